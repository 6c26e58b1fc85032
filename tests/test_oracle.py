"""Pins of the CPU oracle against what the paper and the mathematics fix.

* a hand-derived worked example with the paper's figure parameters
  (T = 5, chunks of 2; Fig. kernel_update, Sections 5.1-5.4);
* a pure-Python brute force of the definition on tiny random streams;
* incremental == static closed form on every batch prefix;
* closed forms for the 1M-point uniform case (node count, split schedule,
  expected voxel count from cell occupancy probabilities);
* invariants (each point stored once, capacities, nesting, chunk counts);
* error behaviour (out-of-cube batch rejected with no change, empty batch,
  iteration cap, unsplittable one-unit leaves).
"""
import math

import numpy as np
import pytest

import oracle
from helpers import (assert_snapshots_equal, brute_force, check_invariants, compare_to_brute,
                     load_golden, pack_rgba, points_array, snapshot_to_dicts)
from paper_2310_03567_gb300 import synth


# ------------------------------------------------------------- worked example

def _golden_stream(g):
    rows, k = [], 0
    for b in g["batches"]:
        batch = []
        for (x, y, z) in b:
            batch.append((x, y, z, k + 1, 2 * (k + 1), 3 * (k + 1), 255 - k))
            k += 1
        rows.append(batch)
    return rows


def _golden_expected(g, exp):
    out = []
    for nd in exp["nodes"]:
        d = {"level": nd["level"], "min": tuple(nd["min"]), "log2size": nd["log2size"],
             "inner": nd["inner"], "n_chunks": nd["n_chunks"]}
        if nd["inner"]:
            d["voxels"] = [(c, tuple(xyz), pack_rgba(w + 1, 2 * (w + 1), 3 * (w + 1), 255 - w))
                           for c, xyz, w in nd["voxels"]]
        else:
            d["points"] = nd["points"]
        out.append(d)
    return out


def _strip(dicts):
    return [{k: v for k, v in d.items() if k != "n"} for d in dicts]


def test_worked_example_incremental_and_static():
    g = load_golden("worked_example.json")
    c = g["config"]
    cfg = oracle.Config.make(root_min=c["root_min"], root_log2=c["root_log2"],
                             leaf_capacity=c["leaf_capacity"], chunk_points=c["chunk_points"],
                             grid_log2=c["grid_log2"])
    batches = _golden_stream(g)
    inc = oracle.Incremental(cfg)
    prefix = []
    for b, exp in zip(batches, g["expected"]):
        assert inc.insert(points_array(b)) == oracle.OK
        prefix += b
        want = _golden_expected(g, exp)
        got = _strip(snapshot_to_dicts(inc.snapshot()))
        assert got == want
        st = inc.stats()
        for k, v in exp["stats"].items():
            assert st[k] == v, (k, st[k], v)
        static = _strip(snapshot_to_dicts(oracle.static_build(cfg, points_array(prefix))))
        assert static == want


# ------------------------------------------------------------------ brute force

def _random_stream(rng, n, root_log2, dup_frac=0.3, cluster=False):
    side = 1 << root_log2
    if cluster:
        centre = rng.integers(0, side, 3)
        xyz = np.clip(centre + rng.integers(-2, 3, (n, 3)), 0, side - 1)
    else:
        xyz = rng.integers(0, side, (n, 3))
    # repeat some positions so that cells and leaves are contested
    nd = int(n * dup_frac)
    if nd and n > 1:
        src = rng.integers(0, n, nd)
        dst = rng.integers(0, n, nd)
        xyz[dst] = xyz[src]
    col = rng.integers(0, 256, (n, 4))
    return [tuple(int(v) for v in xyz[k]) + tuple(int(v) for v in col[k]) for k in range(n)]


def _cuts(rng, n, parts):
    if n == 0:
        return [0]
    cuts = sorted(set(rng.integers(0, n + 1, parts).tolist()) | {0, n})
    return cuts


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(1000 + seed)
    root_log2 = int(rng.integers(2, 6))
    G = int(rng.integers(1, 3))
    T = int(rng.integers(1, 7))
    C = int(rng.integers(1, 4))
    n = int(rng.integers(0, 120))
    rows = _random_stream(rng, n, root_log2, cluster=bool(seed % 3 == 0))
    cfg = oracle.Config.make(root_min=(0, 0, 0), root_log2=root_log2, leaf_capacity=T,
                             chunk_points=C, grid_log2=G)
    stream = [(r[0], r[1], r[2], pack_rgba(*r[3:])) for r in rows]
    inc = oracle.Incremental(cfg)
    cuts = _cuts(rng, n, 4)
    for a, b in zip(cuts[:-1], cuts[1:]):
        assert inc.insert(points_array(rows[a:b])) == oracle.OK
        compare_to_brute(inc.snapshot(), stream[:b], (0, 0, 0), root_log2, T, C, G)
    compare_to_brute(oracle.static_build(cfg, points_array(rows)), stream, (0, 0, 0), root_log2,
                     T, C, G)


def test_brute_force_offset_root_and_boundaries():
    """Negative root minimum, points on the cube's faces and last unit."""
    rng = np.random.default_rng(7)
    root_min, L = (-8, 16, -4), 3
    corners = [(root_min[0] + dx, root_min[1] + dy, root_min[2] + dz)
               for dx in (0, 7) for dy in (0, 7) for dz in (0, 7)]
    rows = []
    for k in range(60):
        x, y, z = corners[k % 8] if k < 24 else tuple(
            int(root_min[a] + rng.integers(0, 8)) for a in range(3))
        rows.append((x, y, z, k, 255 - k, 7, 9))
    cfg = oracle.Config.make(root_min=root_min, root_log2=L, leaf_capacity=3, chunk_points=2,
                             grid_log2=2)
    stream = [(r[0], r[1], r[2], pack_rgba(*r[3:])) for r in rows]
    inc = oracle.Incremental(cfg)
    for a in range(0, 60, 7):
        assert inc.insert(points_array(rows[a:a + 7])) == oracle.OK
    compare_to_brute(inc.snapshot(), stream, root_min, L, 3, 2, 2)


def test_brute_force_pins_paper_grid_cells():
    """Cell and centre formulas at the paper's 128^3 grid, by containment."""
    rng = np.random.default_rng(3)
    G = 7
    for L in (3, 7, 13, 20, 31):
        s = 1 << L
        mn = np.array([-(1 << 30), 5, 1 << 20], np.int64)
        off = rng.integers(0, s, (2000, 3)).astype(np.int64)
        off[:8] = [[0, 0, 0], [s - 1, s - 1, s - 1], [s // 2, 0, 0], [0, s // 2 - 1, 0],
                   [1, 1, 1], [s // 128, 0, 0], [s // 128 - 1, 0, 0], [s - 2, 3, 4]]
        for a in range(3):
            c = (off[:, a] << G) >> L
            # containment: c*s <= off*2^G < (c+1)*s
            assert np.all(c * s <= off[:, a] * (1 << G))
            assert np.all(off[:, a] * (1 << G) < (c + 1) * s)
            centre = mn[a] + (((2 * c + 1) << L) >> (G + 1))
            exact2 = 2 * mn[a] * (1 << G) + (2 * c + 1) * s  # 2^(G+1) * exact centre
            assert np.all(centre * (1 << (G + 1)) <= exact2)
            assert np.all(exact2 < (centre + 1) * (1 << (G + 1)))


# -------------------------------------------------------- incremental vs static

@pytest.mark.parametrize("case", ["uniform", "cluster", "dups"])
def test_incremental_equals_static_on_prefixes(case):
    rng = np.random.default_rng({"uniform": 1, "cluster": 2, "dups": 3}[case])
    L = 12
    n = 40_000
    if case == "uniform":
        pts = synth.uniform(11, 1 << L, n)
    elif case == "cluster":
        pts = synth.uniform(12, 1 << 6, n)
        pts["x"] += 1500
        pts["y"] += 3000
        pts["z"] += 7
    else:
        pts = synth.uniform(13, 1 << L, n)
        idx = rng.integers(0, n, n // 2)
        pts[rng.integers(0, n, n // 2)] = pts[idx]
    cfg = oracle.Config.make(root_log2=L, leaf_capacity=500, chunk_points=37, grid_log2=4)
    inc = oracle.Incremental(cfg)
    cuts = sorted(set(rng.integers(1, n, 9).tolist()) | {n})
    a = 0
    for b in cuts:
        assert inc.insert(pts[a:b]) == oracle.OK
        a = b
        snap = inc.snapshot()
        assert_snapshots_equal(snap, oracle.static_build(cfg, pts[:b]))
        check_invariants(snap, pts[:b], (0, 0, 0), L, 500, 37, 4)
    st = inc.stats()
    assert st["spill_voxels_at_old_inner"] == 0  # re-inserted points add nothing above
    assert st["chunks_live"] + st["chunks_pool"] == st["chunks_bumped"]


def test_batch_partition_independence():
    """The final octree does not depend on how the stream is cut (one batch,
    many batches, single points)."""
    pts = synth.uniform(21, 1 << 10, 3000)
    cfg = oracle.Config.make(root_log2=10, leaf_capacity=40, chunk_points=16, grid_log2=3)
    one, _ = oracle.incremental_build(cfg, [pts])
    many, _ = oracle.incremental_build(cfg, [pts[k:k + 97] for k in range(0, 3000, 97)])
    singles, _ = oracle.incremental_build(cfg, [pts[k:k + 1] for k in range(3000)])
    assert_snapshots_equal(one, many)
    assert_snapshots_equal(one, singles)


# ------------------------------------------------------ uniform 1M closed forms

@pytest.fixture(scope="module")
def uniform_1m():
    w = synth.uniform_workload()
    cfg = oracle.Config.make(root_log2=20)
    inc = oracle.Incremental(cfg)
    nodes_after = []
    for b in w.batches():
        assert inc.insert(b) == oracle.OK
        nodes_after.append(len(inc.snapshot().nodes))
    return w, cfg, inc.snapshot(), inc.stats(), nodes_after


def _expected_occupied(intervals, n):
    """Expected occupied cells when n points fall uniformly; intervals are
    (count, probability) per axis and the three axes are independent."""
    tot = 0.0
    for ca, qa in intervals[0]:
        for cb, qb in intervals[1]:
            for cc, qc in intervals[2]:
                tot += ca * cb * cc * (1.0 - (1.0 - qa * qb * qc) ** n)
    return tot


def test_uniform_1m_structure(uniform_1m):
    w, cfg, snap, st, nodes_after = uniform_1m
    # root (1M > T) and all 8 level-1 nodes (108k-144k > T) split; the 64
    # level-2 nodes hold 9.7k-18k <= T points: 1 + 8 + 64 nodes.
    assert len(snap.nodes) == 73
    assert snap.nodes["is_inner"].sum() == 9
    assert np.all(snap.nodes["level"][:1] == 0) and np.sum(snap.nodes["level"] == 2) == 64
    # Split schedule: the root after 100k points, the level-1 nodes holding more
    # than 1/8 of the points after 400k (4 of them), the rest after 500k.
    assert nodes_after == [9, 9, 9, 41, 73, 73, 73, 73, 73, 73]
    assert st["splits"] == 9
    check_invariants(snap, w.points, (0, 0, 0), 20, 50_000, 1000, 7)


def test_uniform_1m_voxel_count_closed_form(uniform_1m):
    w, cfg, snap, st, _ = uniform_1m
    n = 1_000_000
    # root grid: cells of 8192 mm; [0, 1e6) = 122 full cells + one of 576 mm
    root_axis = [(122, 8192 / 1e6), (1, 576 / 1e6)]
    e_root = _expected_occupied([root_axis] * 3, n)
    # level-1 grids: cells of 4096 mm; lower half 128 full cells, upper half
    # [524288, 1e6) = 116 full cells + one of 576 mm
    lo, hi = [(128, 4096 / 1e6)], [(116, 4096 / 1e6), (1, 576 / 1e6)]
    e_l1 = sum(_expected_occupied([ax, ay, az], n)
               for ax in (lo, hi) for ay in (lo, hi) for az in (lo, hi))
    nv = snap.nodes["n_voxels"].astype(np.int64)
    lvl = snap.nodes["level"]
    tol = lambda e: 6.0 * math.sqrt(e)  # occupancy variance is below the mean
    assert abs(nv[lvl == 0].sum() - e_root) < tol(e_root)
    assert abs(nv[lvl == 1].sum() - e_l1) < tol(e_l1)
    assert st["voxels"] == len(snap.voxels)


def test_uniform_1m_voxel_winners_sampled(uniform_1m):
    """Each sampled voxel's colour is that of the lowest-index point in its
    cell, found by a scan of the whole stream."""
    w, cfg, snap, _, _ = uniform_1m
    pts = w.points
    rgba = (pts["r"].astype(np.uint32) | (pts["g"].astype(np.uint32) << 8) |
            (pts["b"].astype(np.uint32) << 16) | (pts["a"].astype(np.uint32) << 24))
    vo = np.repeat(np.arange(len(snap.nodes)), snap.nodes["n_voxels"].astype(np.int64))
    rng = np.random.default_rng(5)
    for k in rng.choice(len(snap.voxels), 40, replace=False):
        nd = snap.nodes[vo[k]]
        L, mn = int(nd["log2size"]), nd["min"].astype(np.int64)
        cell = int(snap.voxels["cell"][k])
        c = (cell % 128, (cell // 128) % 128, cell // 16384)
        s = 1 << L
        inside = np.ones(len(pts), bool)
        for a, f in enumerate("xyz"):
            d = pts[f].astype(np.int64) - mn[a]
            inside &= (c[a] * s <= d * 128) & (d * 128 < (c[a] + 1) * s)
        first = np.argmax(inside)
        assert inside[first]
        assert rgba[first] == snap.voxels["rgba"][k]


# ------------------------------------------------------------- other workloads

def test_aerial_sample_invariants():
    w = synth.aerial_workload(n=1_500_000, batch=250_000)
    cfg = oracle.Config.make(root_log2=22)
    snap, st = oracle.incremental_build(cfg, w.batches())
    check_invariants(snap, w.points, (0, 0, 0), 22, 50_000, 1000, 7)
    assert_snapshots_equal(snap, oracle.static_build(cfg, w.points))
    assert st["spill_voxels_at_old_inner"] == 0


def test_clustered_sample_invariants():
    w = synth.clustered_workload(n=1_200_000, n_quads=300, batch_lo=50_000, batch_hi=400_000)
    cfg = oracle.Config.make(root_log2=21)
    snap, st = oracle.incremental_build(cfg, w.batches())
    stream = w.stream()
    check_invariants(snap, stream, (0, 0, 0), 21, 50_000, 1000, 7)
    assert_snapshots_equal(snap, oracle.static_build(cfg, stream))
    assert st["chunks_live"] + st["chunks_pool"] == st["chunks_bumped"]


# -------------------------------------------------------------- error handling

def test_out_of_cube_batch_rejected_without_change():
    cfg = oracle.Config.make(root_min=(0, 0, 0), root_log2=4, leaf_capacity=3, chunk_points=2,
                             grid_log2=2)
    inc = oracle.Incremental(cfg)
    good = points_array([(1, 2, 3, 1, 1, 1, 1), (4, 5, 6, 2, 2, 2, 2), (9, 9, 9, 3, 3, 3, 3),
                         (15, 15, 15, 4, 4, 4, 4)])
    assert inc.insert(good) == oracle.OK
    before = inc.snapshot()
    for bad_xyz in [(16, 0, 0), (0, -1, 0), (0, 0, 1 << 20)]:
        bad = points_array([(1, 1, 1, 0, 0, 0, 0), bad_xyz + (0, 0, 0, 0)])
        assert inc.insert(bad) == oracle.ERR_OUT_OF_BOUNDS
        assert_snapshots_equal(inc.snapshot(), before)
    assert inc.insert(points_array([])) == oracle.OK
    assert_snapshots_equal(inc.snapshot(), before)
    # arrival indices continue after the rejected batches
    assert inc.insert(points_array([(2, 2, 2, 5, 5, 5, 5)])) == oracle.OK
    assert sorted(inc.snapshot().points["gidx"].tolist()) == [0, 1, 2, 3, 4]


def test_unsplittable_one_unit_leaf():
    """More than T identical points: nodes split down to side 1, which keeps them."""
    cfg = oracle.Config.make(root_log2=3, leaf_capacity=4, chunk_points=3, grid_log2=1)
    rows = [(5, 2, 7, k, k, k, 255) for k in range(11)] + [(0, 0, 0, 9, 9, 9, 9)]
    snap, st = oracle.incremental_build(cfg, [points_array(rows[:6]), points_array(rows[6:])])
    leaf = snap.nodes[(snap.nodes["is_inner"] == 0) & (snap.nodes["n_points"] > 0)]
    big = leaf[leaf["n_points"] == 11]
    assert len(big) == 1 and big["log2size"][0] == 0 and big["n_chunks"][0] == 4
    stream = [(r[0], r[1], r[2], pack_rgba(*r[3:])) for r in rows]
    compare_to_brute(snap, stream, (0, 0, 0), 3, 4, 3, 1)


def test_iteration_cap():
    cfg = oracle.Config.make(root_log2=10, leaf_capacity=2, chunk_points=2, grid_log2=2,
                             max_expand_iters=2)
    inc = oracle.Incremental(cfg)
    rows = [(512 + k % 3, 512, 512, 1, 1, 1, 1) for k in range(10)]
    assert inc.insert(points_array(rows)) == oracle.ERR_ITER_CAP


def test_brute_force_helper_self_check():
    """The brute force agrees with a hand count on a two-point stream."""
    stream = [(0, 0, 0, 7), (3, 3, 3, 9)]
    out = brute_force(stream, (0, 0, 0), 2, 1, 1, 1)
    assert [d["level"] for d in out] == [0] + [1] * 8
    assert out[0]["voxels"] == [(0, (1, 1, 1), 7), (7, (3, 3, 3), 9)]
    assert out[1]["points"] == [0] and out[-1]["points"] == [1]
