"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Octree results are integers, so the bar is bit-exact: canonical node set,
per-node voxel sets (cell, position, rgba) and per-leaf point multisets
(x, y, z, rgba, gidx) must equal the oracle's byte for byte, after every batch
on the small cases and at the end on the large ones.
"""
import zlib

import numpy as np
import pytest

import oracle
from helpers import (assert_snapshots_equal, check_allocator, check_invariants, compare_to_brute,
                     load_golden, pack_rgba, points_array)
from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def make_tree(data_bytes=256 << 20, **kw):
    cfg = simlod.default_config(**kw)
    arena = simlod.make_arena(cfg, data_bytes)
    return simlod.Octree(cfg, arena, stream=torch.cuda.Stream())


def small_caps(**kw):
    base = dict(max_batch_points=1 << 20, spill_capacity=1 << 20, backlog_capacity=1 << 20,
                max_nodes=1 << 16)
    base.update(kw)
    return base


def oracle_cfg(**kw):
    keep = {k: kw[k] for k in ("root_min", "root_log2", "leaf_capacity", "chunk_points",
                               "grid_log2") if k in kw}
    return oracle.Config.make(**keep)


def same(a, b):
    assert_snapshots_equal(a, b)


# ------------------------------------------------------------------ golden

def test_worked_example_on_gpu():
    g = load_golden("worked_example.json")
    c = g["config"]
    kw = dict(root_min=c["root_min"], root_log2=c["root_log2"], leaf_capacity=c["leaf_capacity"],
              chunk_points=c["chunk_points"], grid_log2=c["grid_log2"])
    tree = make_tree(16 << 20, **small_caps(**kw))
    ref = oracle.Incremental(oracle_cfg(**kw))
    k = 0
    for b in g["batches"]:
        rows = []
        for (x, y, z) in b:
            rows.append((x, y, z, k + 1, 2 * (k + 1), 3 * (k + 1), 255 - k))
            k += 1
        pts = points_array(rows)
        tree.insert(simlod.points_tensor(pts))
        assert ref.insert(pts) == oracle.OK
        same(tree.snapshot(), ref.snapshot())
    st = tree.stats()
    assert st["splits"] == 2 and st["spilled"] == 5 and st["voxels"] == 15


# -------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(10))
def test_tiny_random_against_brute_force(seed):
    rng = np.random.default_rng(2000 + seed)
    L = int(rng.integers(2, 7))
    G = int(rng.integers(1, 4))
    T = int(rng.integers(1, 9))
    C = int(rng.integers(1, 5))
    n = int(rng.integers(1, 200))
    side = 1 << L
    if seed % 3 == 0:
        xyz = np.clip(rng.integers(0, side, 3) + rng.integers(-2, 3, (n, 3)), 0, side - 1)
    else:
        xyz = rng.integers(0, side, (n, 3))
    dup = rng.integers(0, n, n // 3)
    xyz[rng.integers(0, n, n // 3)] = xyz[dup]
    col = rng.integers(0, 256, (n, 4))
    rows = [tuple(int(v) for v in xyz[k]) + tuple(int(v) for v in col[k]) for k in range(n)]
    kw = dict(root_log2=L, leaf_capacity=T, chunk_points=C, grid_log2=G)
    tree = make_tree(64 << 20, **small_caps(**kw))
    ref = oracle.Incremental(oracle_cfg(**kw))
    cuts = sorted(set(rng.integers(0, n + 1, 5).tolist()) | {0, n})
    stream = [(r[0], r[1], r[2], pack_rgba(*r[3:])) for r in rows]
    for a, b in zip(cuts[:-1], cuts[1:]):
        pts = points_array(rows[a:b])
        if b > a:
            tree.insert(simlod.points_tensor(pts))
        assert ref.insert(pts) == oracle.OK
        snap = tree.snapshot()
        same(snap, ref.snapshot())
    compare_to_brute(tree.snapshot(), stream, (0, 0, 0), L, T, C, G)


# ------------------------------------------------------- randomized configs

CASES = [
    # (name, root_log2, T, C, G, n, batches, generator)
    ("uniform_mid", 16, 300, 50, 5, 200_000, 7, "uniform"),
    ("uniform_ragged", 14, 1000, 1, 3, 77_777, 5, "uniform"),
    ("cluster_deep", 20, 64, 17, 7, 120_000, 4, "cluster"),
    ("dups", 12, 100, 1000, 7, 150_000, 6, "dups"),
    ("big_chunks", 18, 5000, 4096, 6, 300_000, 3, "uniform"),
    ("single_leaf", 18, 50_000, 1000, 7, 40_000, 4, "uniform"),
]


def _gen(kind, n, L, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return synth.uniform(seed, 1 << L, n)
    if kind == "cluster":
        pts = synth.uniform(seed, 1 << 9, n)
        pts["x"] += 70_000
        pts["y"] += 300_000
        pts["z"] += 1_000
        return pts
    pts = synth.uniform(seed, 1 << L, n)
    pts[rng.integers(0, n, n // 2)] = pts[rng.integers(0, n, n // 2)]
    return pts


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_random_configs_every_batch(case):
    name, L, T, C, G, n, nb, kind = case
    pts = _gen(kind, n, L, zlib.crc32(name.encode()) % 1000)
    rng = np.random.default_rng(len(name))
    cuts = sorted(set(rng.integers(1, n, nb - 1).tolist()) | {0, n})
    kw = dict(root_log2=L, leaf_capacity=T, chunk_points=C, grid_log2=G)
    tree = make_tree(1 << 30, **small_caps(**kw))
    ref = oracle.Incremental(oracle_cfg(**kw))
    for a, b in zip(cuts[:-1], cuts[1:]):
        tree.insert(simlod.points_tensor(pts[a:b]))
        assert ref.insert(pts[a:b]) == oracle.OK
        same(tree.snapshot(), ref.snapshot())
    snap = tree.snapshot()
    check_invariants(snap, pts, (0, 0, 0), L, T, C, G)
    st = tree.stats()
    assert st["points"] == n and st["batches"] == len(cuts) - 1
    check_allocator(snap, st)


# -------------------------------------------------------- paper-size cases

def test_uniform_1m_every_batch():
    """1M uniform points in a 1 km cube, 10 batches of 100k, T = 50k, 128^3."""
    w = synth.uniform_workload()
    tree = make_tree(1 << 30, root_log2=20, max_batch_points=1 << 20)
    ref = oracle.Incremental(oracle.Config.make(root_log2=20))
    nodes_after = []
    for b in w.batches():
        tree.insert(simlod.points_tensor(b))
        assert ref.insert(b) == oracle.OK
        snap = tree.snapshot()
        same(snap, ref.snapshot())
        nodes_after.append(len(snap.nodes))
    assert nodes_after == [9, 9, 9, 41, 73, 73, 73, 73, 73, 73]


def test_aerial_prefix_bit_exact():
    w = synth.aerial_workload(n=6_000_000)
    tree = make_tree(4 << 30, root_log2=22)
    for b in w.batches():
        tree.insert(simlod.points_tensor(b))
    snap = tree.snapshot()
    check_allocator(snap, tree.stats())
    same(snap, oracle.static_build(oracle.Config.make(root_log2=22), w.points))


def test_clustered_sample_bit_exact():
    w = synth.clustered_workload(n=8_000_000, n_quads=600, batch_lo=200_000, batch_hi=2_000_000)
    tree = make_tree(4 << 30, root_log2=21)
    for b in w.batches():
        tree.insert(simlod.points_tensor(b))
    snap = tree.snapshot()
    same(snap, oracle.static_build(oracle.Config.make(root_log2=21), w.stream()))
    st = tree.stats()
    assert st["spilled"] > 0 and st["splits"] > 0


# ------------------------------------------------------------------ edges

def test_empty_batches_and_rejection_leave_state_unchanged():
    kw = dict(root_min=(-100, 0, 50), root_log2=10, leaf_capacity=20, chunk_points=8, grid_log2=3)
    tree = make_tree(64 << 20, **small_caps(**kw))
    ref = oracle.Incremental(oracle_cfg(**kw))
    pts = synth.uniform(5, 1 << 10, 500)
    pts["x"] -= 100
    pts["z"] += 50
    tree.insert(simlod.points_tensor(pts[:300]))
    assert ref.insert(pts[:300]) == oracle.OK
    before = tree.snapshot()
    assert tree.insert(simlod.points_tensor(pts[:0]), check=False) == simlod.OK
    for bad in ((924, 0, 50), (-101, 5, 60), (0, 0, 49), (0, 1 << 10, 60)):
        b = pts[300:340].copy()
        b[17] = bad + (1, 2, 3, 4)
        assert tree.insert(simlod.points_tensor(b), check=False) == simlod.ERR_OUT_OF_BOUNDS
        same(tree.snapshot(), before)
    tree.insert(simlod.points_tensor(pts[300:]))
    assert ref.insert(pts[300:]) == oracle.OK
    same(tree.snapshot(), ref.snapshot())
    assert tree.stats()["rejected_batches"] == 4


def test_boundary_points_and_unsplittable_leaf():
    kw = dict(root_log2=5, leaf_capacity=4, chunk_points=3, grid_log2=2)
    rows = [(31, 31, 31, 1, 1, 1, 1)] * 9 + [(0, 0, 0, 2, 2, 2, 2)] * 3 + \
           [(16, 15, 16, k, k, k, k) for k in range(7)]
    tree = make_tree(16 << 20, **small_caps(**kw))
    ref = oracle.Incremental(oracle_cfg(**kw))
    for a in range(0, len(rows), 5):
        pts = points_array(rows[a:a + 5])
        tree.insert(simlod.points_tensor(pts))
        assert ref.insert(pts) == oracle.OK
    same(tree.snapshot(), ref.snapshot())


def test_single_point_batches_and_partition_independence():
    pts = synth.uniform(9, 1 << 8, 700)
    kw = dict(root_log2=8, leaf_capacity=10, chunk_points=4, grid_log2=3)
    one = make_tree(64 << 20, **small_caps(**kw))
    one.insert(simlod.points_tensor(pts))
    singles = make_tree(64 << 20, **small_caps(**kw))
    for k in range(len(pts)):
        singles.insert(simlod.points_tensor(pts[k:k + 1]))
    same(one.snapshot(), singles.snapshot())
    same(one.snapshot(), oracle.static_build(oracle_cfg(**kw), pts))


def test_max_batch_size_and_determinism():
    n = 1 << 20
    pts = synth.uniform(17, 1 << 18, n)
    kw = dict(root_log2=18, leaf_capacity=2000, chunk_points=100, grid_log2=6,
              max_batch_points=n, backlog_capacity=4 << 20)
    a = make_tree(1 << 30, **small_caps(**kw))
    b = make_tree(1 << 30, **small_caps(**kw))
    a.insert(simlod.points_tensor(pts))
    b.insert(simlod.points_tensor(pts))
    same(a.snapshot(), b.snapshot())
    assert b.insert(simlod.points_tensor(synth.uniform(1, 8, n + 1)), check=False) == \
        simlod.ERR_INVALID_ARG


def test_host_insert_matches_device_insert():
    pts = synth.uniform(23, 1 << 16, 90_000)
    kw = dict(root_log2=16, leaf_capacity=800, chunk_points=64, grid_log2=5)
    d = make_tree(256 << 20, **small_caps(**kw))
    h = make_tree(256 << 20, **small_caps(**kw))
    for lo in range(0, len(pts), 30_000):
        d.insert(simlod.points_tensor(pts[lo:lo + 30_000]))
        h.insert_host(pts[lo:lo + 30_000])
    same(d.snapshot(), h.snapshot())


def test_reset_rebuilds_identically():
    pts = synth.uniform(29, 1 << 16, 50_000)
    kw = dict(root_log2=16, leaf_capacity=500, chunk_points=50, grid_log2=6)
    t = make_tree(256 << 20, **small_caps(**kw))
    t.insert(simlod.points_tensor(pts))
    first = t.snapshot()
    t.reset()
    assert len(t.snapshot().nodes) == 1
    t.insert(simlod.points_tensor(pts))
    same(t.snapshot(), first)


def test_frame_budget_stops_between_batches():
    pts = synth.uniform(31, 1 << 16, 40_000)
    kw = dict(root_log2=16, leaf_capacity=500, chunk_points=50, grid_log2=6)
    t = make_tree(256 << 20, **small_caps(**kw))
    batches = [simlod.points_tensor(pts[k:k + 10_000]) for k in range(0, 40_000, 10_000)]
    rc, used = t.frame_update(batches, budget_ns=0)
    assert rc == simlod.OK and used == 1  # the budget is checked before batch 2
    rc, used2 = t.frame_update(batches[used:], budget_ns=10**12)
    assert rc == simlod.OK and used + used2 == 4
    same(t.snapshot(), oracle.static_build(oracle_cfg(**kw), pts))


# --------------------------------------------------- injected capacity errors

@pytest.mark.parametrize("what", ["arena", "nodes", "spill", "backlog", "iters"])
def test_capacity_errors_poison_the_handle(what):
    # 20k-point batches into T = 200 leaves: the first batch builds leaves of
    # ~40 points, which refill and split (spilling ~200 points each) by batch 6
    pts = synth.uniform(37, 1 << 16, 200_000)
    kw = small_caps(root_log2=16, leaf_capacity=200, chunk_points=16, grid_log2=7)
    data = 256 << 20
    expect = {"arena": simlod.ERR_ARENA_FULL, "nodes": simlod.ERR_NODES_FULL,
              "spill": simlod.ERR_SPILL_FULL, "backlog": simlod.ERR_BACKLOG_FULL,
              "iters": simlod.ERR_ITER_CAP}[what]
    if what == "arena":
        data = 2 << 20
    elif what == "nodes":
        kw["max_nodes"] = 64
    elif what == "spill":
        kw["spill_capacity"] = 100
    elif what == "backlog":
        kw["backlog_capacity"] = 1000
    else:
        kw["max_expand_iters"] = 1
    t = make_tree(data, **kw)
    rc = simlod.OK
    for lo in range(0, len(pts), 20_000):
        rc = t.insert(simlod.points_tensor(pts[lo:lo + 20_000]), check=False)
        if rc != simlod.OK:
            break
    assert rc == expect
    assert t.insert(simlod.points_tensor(pts[:10]), check=False) == simlod.ERR_POISONED
    assert t.stats()["sticky_status"] == expect
    t.reset()
    small = pts[:100]
    t.insert(simlod.points_tensor(small))
    same(t.snapshot(), oracle.static_build(oracle_cfg(**kw), small))
