"""GPU parity of the fused form (one persistent cooperative launch over a list
of batches, grid barriers between phases) against the CPU oracle.

Each batch is still one complete update, so the octree after every launch
must equal the oracle's after the same batches, byte for byte; a launch over
many batches must equal one launch per batch, the plain per-kernel path and
the static closed form.
"""
import numpy as np
import pytest

import oracle
from helpers import (assert_snapshots_equal, check_allocator, check_invariants, load_golden,
                     points_array)
from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def make_tree(data_bytes=256 << 20, **kw):
    cfg = simlod.default_config(**kw)
    arena = simlod.make_arena(cfg, data_bytes)
    return simlod.Octree(cfg, arena, stream=torch.cuda.Stream())


def caps(**kw):
    base = dict(max_batch_points=1 << 20, spill_capacity=1 << 20, backlog_capacity=1 << 21,
                max_nodes=1 << 16)
    base.update(kw)
    return base


def ocfg(**kw):
    keep = {k: kw[k] for k in ("root_min", "root_log2", "leaf_capacity", "chunk_points",
                               "grid_log2") if k in kw}
    return oracle.Config.make(**keep)


def fused_insert(tree, arrays):
    ts = [simlod.points_tensor(a) for a in arrays]
    tree.insert_many(ts)
    return tree.sync()


def test_worked_example_fused_each_and_all():
    g = load_golden("worked_example.json")
    c = g["config"]
    kw = dict(root_min=c["root_min"], root_log2=c["root_log2"], leaf_capacity=c["leaf_capacity"],
              chunk_points=c["chunk_points"], grid_log2=c["grid_log2"])
    batches, k = [], 0
    for b in g["batches"]:
        rows = []
        for (x, y, z) in b:
            rows.append((x, y, z, k + 1, 2 * (k + 1), 3 * (k + 1), 255 - k))
            k += 1
        batches.append(points_array(rows))
    each = make_tree(16 << 20, **caps(**kw))
    ref = oracle.Incremental(ocfg(**kw))
    for b in batches:
        assert fused_insert(each, [b]) == simlod.OK
        assert ref.insert(b) == oracle.OK
        assert_snapshots_equal(each.snapshot(), ref.snapshot())
    both = make_tree(16 << 20, **caps(**kw))
    assert fused_insert(both, batches) == simlod.OK
    assert_snapshots_equal(both.snapshot(), ref.snapshot())
    st = both.stats()
    assert st["batches"] == 2 and st["splits"] == 2 and st["spilled"] == 5


CASES = [
    ("uniform_mid", 16, 300, 50, 5, 200_000, 9, "uniform"),
    ("ragged_c1", 14, 1000, 1, 3, 77_777, 5, "uniform"),
    ("cluster_deep", 20, 64, 17, 7, 120_000, 6, "cluster"),
    ("dups", 12, 100, 1000, 7, 150_000, 6, "dups"),
    ("tiny_T", 10, 3, 2, 2, 20_000, 11, "uniform"),
]


def _gen(kind, n, L, seed):
    rng = np.random.default_rng(seed)
    if kind == "cluster":
        pts = synth.uniform(seed, 1 << 9, n)
        pts["x"] += 70_000
        pts["y"] += 300_000
        pts["z"] += 1_000
        return pts
    pts = synth.uniform(seed, 1 << L, n)
    if kind == "dups":
        pts[rng.integers(0, n, n // 2)] = pts[rng.integers(0, n, n // 2)]
    return pts


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fused_matches_oracle_per_launch_and_in_one_launch(case):
    name, L, T, C, G, n, nb, kind = case
    pts = _gen(kind, n, L, 7 + len(name))
    rng = np.random.default_rng(len(name) * 31)
    cuts = sorted(set(rng.integers(1, n, nb - 1).tolist()) | {0, n})
    parts = [pts[a:b] for a, b in zip(cuts[:-1], cuts[1:])]
    kw = dict(root_log2=L, leaf_capacity=T, chunk_points=C, grid_log2=G)
    per = make_tree(1 << 30, **caps(**kw))
    ref = oracle.Incremental(ocfg(**kw))
    for part in parts:
        assert fused_insert(per, [part]) == simlod.OK
        assert ref.insert(part) == oracle.OK
        assert_snapshots_equal(per.snapshot(), ref.snapshot())
    one = make_tree(1 << 30, **caps(**kw))
    assert fused_insert(one, parts) == simlod.OK
    snap = one.snapshot()
    assert_snapshots_equal(snap, ref.snapshot())
    check_invariants(snap, pts, (0, 0, 0), L, T, C, G)


def test_uniform_1m_one_launch():
    w = synth.uniform_workload()
    tree = make_tree(1 << 30, root_log2=20, max_batch_points=1 << 20)
    assert fused_insert(tree, list(w.batches())) == simlod.OK
    snap = tree.snapshot()
    assert len(snap.nodes) == 73
    assert_snapshots_equal(snap, oracle.static_build(oracle.Config.make(root_log2=20), w.points))


def test_aerial_and_clustered_one_launch():
    w = synth.aerial_workload(n=6_000_000)
    t = make_tree(4 << 30, root_log2=22)
    assert fused_insert(t, list(w.batches())) == simlod.OK
    snap = t.snapshot()
    check_allocator(snap, t.stats())
    assert_snapshots_equal(snap, oracle.static_build(oracle.Config.make(root_log2=22), w.points))
    w = synth.clustered_workload(n=8_000_000, n_quads=600, batch_lo=200_000, batch_hi=2_000_000)
    t = make_tree(4 << 30, root_log2=21)
    assert fused_insert(t, list(w.batches())) == simlod.OK
    snap = t.snapshot()
    check_allocator(snap, t.stats())
    assert_snapshots_equal(snap, oracle.static_build(oracle.Config.make(root_log2=21), w.stream()))


def test_rejected_batch_inside_a_launch_is_skipped():
    kw = dict(root_log2=12, leaf_capacity=50, chunk_points=8, grid_log2=4)
    pts = synth.uniform(3, 1 << 12, 4000)
    bad = pts[1000:1500].copy()
    bad[123] = (5000, 1, 1, 0, 0, 0, 0)
    t = make_tree(64 << 20, **caps(**kw))
    rc = fused_insert(t, [pts[:1000], bad, pts[1000:4000], pts[:0]])
    assert rc == simlod.ERR_OUT_OF_BOUNDS
    assert t.sync() == simlod.OK  # reported once
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts))
    st = t.stats()
    assert st["rejected_batches"] == 1 and st["batches"] == 2


def test_fused_frame_budget():
    kw = dict(root_log2=16, leaf_capacity=500, chunk_points=50, grid_log2=6)
    pts = synth.uniform(31, 1 << 16, 40_000)
    t = make_tree(256 << 20, **caps(**kw))
    ts = [simlod.points_tensor(pts[k:k + 10_000]) for k in range(0, 40_000, 10_000)]
    rc, used = t.frame_update(ts, budget_ns=0)
    assert rc == simlod.OK and used == 1
    rc, used2 = t.frame_update(ts[used:], budget_ns=10**12)
    assert rc == simlod.OK and used + used2 == 4
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts))


def test_mixing_plain_and_fused_on_one_handle():
    kw = dict(root_log2=16, leaf_capacity=400, chunk_points=32, grid_log2=5)
    pts = synth.uniform(41, 1 << 16, 120_000)
    t = make_tree(512 << 20, **caps(**kw))
    t.insert(simlod.points_tensor(pts[:30_000]))
    assert fused_insert(t, [pts[30_000:50_000], pts[50_000:70_000]]) == simlod.OK
    t.insert(simlod.points_tensor(pts[70_000:100_000]))
    assert fused_insert(t, [pts[100_000:]]) == simlod.OK
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts))


@pytest.mark.parametrize("what", ["arena", "nodes", "spill", "backlog", "iters"])
def test_fused_capacity_errors_poison(what):
    pts = synth.uniform(37, 1 << 16, 200_000)
    kw = caps(root_log2=16, leaf_capacity=200, chunk_points=16, grid_log2=7)
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
    rc = fused_insert(t, [pts[k:k + 20_000] for k in range(0, len(pts), 20_000)])
    assert rc == expect
    assert t.insert(simlod.points_tensor(pts[:10]), check=False) == simlod.ERR_POISONED
    t.reset()
    assert fused_insert(t, [pts[:100]]) == simlod.OK
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts[:100]))


def test_fused_reads_batches_from_pinned_host_memory():
    """Host ingest without a staging copy: the persistent kernel reads the
    batches from pinned host memory over the CPU-GPU link."""
    w = synth.aerial_workload(n=3_000_000)
    host = torch.from_numpy(np.ascontiguousarray(w.points).view(np.uint8).reshape(-1, 16))
    host = host.pin_memory()
    t = make_tree(1 << 30, root_log2=22)
    ptrs = [host.data_ptr() + int(o) * 16 for o in w.offsets]
    assert t.insert_many_ptrs(ptrs, [int(c) for c in w.counts]) == simlod.OK
    assert t.sync() == simlod.OK
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=22), w.points))


def test_morton_ordered_stream():
    """The Morton-ordered input variant (dense, strongly local batches)."""
    w = synth.morton_workload(synth.clustered_workload(n=4_000_000, n_quads=300,
                                                       batch_lo=200_000, batch_hi=1_000_000))
    t = make_tree(2 << 30, root_log2=21)
    assert fused_insert(t, list(w.batches())) == simlod.OK
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=21), w.stream()))


def pinned_batches(w):
    host = torch.from_numpy(np.ascontiguousarray(w.points).view(np.uint8).reshape(-1, 16))
    host = host.pin_memory()
    return host, [host[int(o):int(o) + int(c)] for o, c in zip(w.offsets, w.counts)]


@pytest.mark.parametrize("same_stream", [False, True])
def test_host_fed_launch_waits_for_each_copy(same_stream):
    """Host ingest pipeline: batches copied on a copy stream, the persistent
    launch starts each batch once its ready flag is set."""
    w = synth.aerial_workload(n=4_000_000)
    host, parts = pinned_batches(w)
    t = make_tree(1 << 30, root_log2=22)
    dst = torch.empty_like(host, device="cuda")
    ready = torch.empty(len(parts), dtype=torch.int32, device="cuda")
    cs = t.stream if same_stream else torch.cuda.Stream()
    t.insert_many_host(parts, dst, ready, cs)
    assert t.sync() == simlod.OK
    torch.cuda.synchronize()
    assert int(ready.min().item()) == 1
    check_allocator(t.snapshot(), t.stats())
    assert torch.equal(dst.cpu(), host)
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=22), w.points))
    # a second stream through the same buffers continues the octree
    t.insert_many_host(parts[:2], dst, ready, cs)
    assert t.sync() == simlod.OK
    both = np.concatenate([w.points, w.points[: int(w.offsets[2])]])
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=22), both))


def test_host_fed_launch_rejects_a_batch_outside_the_root():
    kw = dict(root_log2=12, leaf_capacity=50, chunk_points=8, grid_log2=4)
    pts = synth.uniform(3, 1 << 12, 4000)
    bad = pts[1000:1500].copy()
    bad[7] = (1, 1, -3, 0, 0, 0, 0)
    arrays = [pts[:1000], bad, pts[1000:4000], pts[:0]]
    host = [torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1, 16)).pin_memory()
            for a in arrays]
    t = make_tree(64 << 20, **caps(**kw))
    dst = torch.empty((sum(len(a) for a in arrays), 16), dtype=torch.uint8, device="cuda")
    ready = torch.empty(len(arrays), dtype=torch.int32, device="cuda")
    t.insert_many_host(host, dst, ready, torch.cuda.Stream())
    assert t.sync() == simlod.ERR_OUT_OF_BOUNDS
    assert t.sync() == simlod.OK
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts))


def test_host_fed_launch_times_out_on_a_flag_that_is_not_set():
    """A ready flag that stays clear (the copy stream is held by a host
    function for 3 s) ends the launch after the 2 s wait limit with a TIMEOUT
    status; the GPU stays usable and a reset handle works again."""
    import ctypes
    import time

    libcuda = ctypes.CDLL("libcuda.so.1")
    hostfn = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
    hold = hostfn(lambda _: time.sleep(3.0))
    w = synth.aerial_workload(n=2_000_000)
    host, parts = pinned_batches(w)
    t = make_tree(1 << 30, root_log2=22)
    dst = torch.empty_like(host, device="cuda")
    ready = torch.empty(len(parts), dtype=torch.int32, device="cuda")
    cs = torch.cuda.Stream()
    assert libcuda.cuLaunchHostFunc(ctypes.c_void_p(cs.cuda_stream), hold, None) == 0
    t.insert_many_host(parts, dst, ready, cs)
    assert t.sync() == simlod.ERR_TIMEOUT
    assert t.insert(simlod.points_tensor(w.points[:10]), check=False) == simlod.ERR_POISONED
    assert libcuda.cuStreamSynchronize(ctypes.c_void_p(cs.cuda_stream)) == 0
    t.reset()
    t.insert_many_host(parts, dst, ready, cs)
    assert t.sync() == simlod.OK
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=22), w.points))


def test_most_batches_per_launch_and_one_more():
    """16,384 batches in one launch (the limit; most of them a single point,
    some empty) give the oracle's octree; 16,385 are refused with
    INVALID_ARG before anything is enqueued."""
    kw = dict(root_log2=16, leaf_capacity=300, chunk_points=40, grid_log2=5)
    n_b = 16_384
    rng = np.random.default_rng(5)
    sizes = rng.choice([0, 1, 1, 1, 2, 7], n_b)
    pts = synth.uniform(17, 1 << 16, int(sizes.sum()))
    t = make_tree(256 << 20, **caps(**kw))
    dev = simlod.points_tensor(pts)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    ptrs = [dev.data_ptr() + int(o) * 16 for o in offs]
    assert t.insert_many_ptrs(ptrs + ptrs[:1], [int(c) for c in sizes] + [1]) == \
        simlod.ERR_INVALID_ARG
    assert t.insert_many_ptrs(ptrs, [int(c) for c in sizes]) == simlod.OK
    assert t.sync() == simlod.OK
    st = t.stats()
    assert st["points"] == len(pts) and st["batches"] == int((sizes > 0).sum())
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), pts))


def test_grid_barrier_times_out_with_every_block_present():
    """A grid-barrier limit of 1 ns on an ordinary launch (every block is
    resident and arrives, so nothing can hang): the first block that has to
    wait gives up after its first few polls, the launch ends with a TIMEOUT
    status, the handle is poisoned, and a reset handle with the default limit
    builds the oracle's octree again."""
    w = synth.aerial_workload(n=4_000_000)
    dev = simlod.points_tensor(w.points)
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    t = make_tree(1 << 30, root_log2=22)
    t.set_wait_limits(barrier_ns=1)
    rc = simlod.OK
    for _ in range(5):  # a launch whose every barrier completes in a few polls would pass
        t.reset()
        assert t.insert_many_ptrs(ptrs, counts) == simlod.OK
        rc = t.sync()
        if rc != simlod.OK:
            break
    assert rc == simlod.ERR_TIMEOUT
    assert t.stats()["sticky_status"] == simlod.ERR_TIMEOUT
    assert t.insert(simlod.points_tensor(w.points[:10]), check=False) == simlod.ERR_POISONED
    t.set_wait_limits()  # back to the default limits
    t.reset()
    assert t.insert_many_ptrs(ptrs, counts) == simlod.OK
    assert t.sync() == simlod.OK
    assert_snapshots_equal(t.snapshot(),
                           oracle.static_build(oracle.Config.make(root_log2=22), w.points))


def test_progress_counts_finished_batches():
    """simlod_progress: the persistent launch counts the batches it has
    finished in host memory. The count rises batch by batch while a launch
    runs and reaches the batches handed over when it ends; a rejected batch
    counts as finished; batches that a frame budget left out are not counted
    as handed over (in the blocking and the asynchronous form); plain inserts
    change neither count."""
    import time
    kw = dict(root_log2=16, leaf_capacity=500, chunk_points=50, grid_log2=6)
    pts = synth.uniform(51, 1 << 16, 300_000)
    t = make_tree(512 << 20, **caps(**kw))
    assert t.progress() == (0, 0)
    ts = [simlod.points_tensor(pts[k:k + 5_000]) for k in range(0, 200_000, 5_000)]
    torch.cuda.synchronize()
    t.insert_many(ts)
    seen, deadline = [], time.perf_counter() + 60.0
    while time.perf_counter() < deadline:
        fin, sub = t.progress()
        seen.append(fin)
        if fin == sub:
            break
    assert t.sync() == simlod.OK
    assert t.progress() == (40, 40) and seen[-1] == 40
    assert all(a <= b for a, b in zip(seen, seen[1:]))
    assert len(set(seen)) >= 3  # counts between 0 and 40 were seen while the launch ran
    bad = pts[200_000:201_000].copy()
    bad[7] = (200_000, 1, 1, 0, 0, 0, 0)
    rc = fused_insert(t, [pts[201_000:210_000], bad, pts[210_000:220_000]])
    assert rc == simlod.ERR_OUT_OF_BOUNDS and t.sync() == simlod.OK
    assert t.progress() == (43, 43)
    rest = [simlod.points_tensor(pts[k:k + 10_000]) for k in range(220_000, 260_000, 10_000)]
    rc, used = t.frame_update(rest, budget_ns=0)
    assert rc == simlod.OK and used == 1 and t.progress() == (44, 44)
    assert t.insert(simlod.points_tensor(pts[230_000:260_000])) == simlod.OK
    assert t.progress() == (44, 44)
    # the asynchronous frame budget: one batch, the rest dropped, then passed again
    more = [simlod.points_tensor(pts[k:k + 10_000]) for k in range(260_000, 300_000, 10_000)]
    ptrs, cnts = [m.data_ptr() for m in more], [10_000] * 4
    torch.cuda.synchronize()  # raw pointers: the copies must be done before the launch
    assert t.insert_many_ptrs(ptrs, cnts, budget_ns=0) == simlod.OK
    assert t.sync() == simlod.OK and t.progress() == (45, 45)
    assert t.insert_many_ptrs(ptrs[1:], cnts[1:], budget_ns=10**12) == simlod.OK
    assert t.sync() == simlod.OK and t.progress() == (48, 48)
    want = np.concatenate([pts[:200_000], pts[201_000:]])
    assert_snapshots_equal(t.snapshot(), oracle.static_build(ocfg(**kw), want))
