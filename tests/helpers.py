"""Shared test helpers: golden fixtures, a pure-Python brute force of the
octree definition, invariant checks and snapshot comparison.

The brute force restates the octree from geometric containment alone (a point
is in a cube or a cell iff its coordinate lies in the half-open interval), so
it pins the oracle's shift-based cell, octant and centre formulas to their
definitions (Sections 3.1, 3.3, 5.1, 5.2).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def pack_rgba(r, g, b, a) -> int:
    return int(r) | (int(g) << 8) | (int(b) << 16) | (int(a) << 24)


def points_array(xyz_rgba) -> np.ndarray:
    from paper_2310_03567_gb300.synth import POINT_DTYPE
    a = np.zeros(len(xyz_rgba), POINT_DTYPE)
    for k, (x, y, z, r, g, b, al) in enumerate(xyz_rgba):
        a[k] = (x, y, z, r, g, b, al)
    return a


def rgba_of(pts: np.ndarray) -> np.ndarray:
    return (pts["r"].astype(np.uint32) | (pts["g"].astype(np.uint32) << 8) |
            (pts["b"].astype(np.uint32) << 16) | (pts["a"].astype(np.uint32) << 24))


# ----------------------------------------------------------------- brute force

def brute_force(stream, root_min, root_log2, T, C, G):
    """Canonical octree of a point stream, from the definition only.

    ``stream`` is a list of (x, y, z, rgba) in arrival order; returns a list of
    node dicts in canonical order (level, ix, iy, iz) with their points (gidx
    sorted) or voxels (cell sorted). Pure Python: tiny inputs only.
    """
    out = []
    side_cells = 1 << G

    def visit(level, ix, iy, iz):
        L = root_log2 - level
        s = 1 << L
        mn = (root_min[0] + ix * s, root_min[1] + iy * s, root_min[2] + iz * s)
        members = [g for g, p in enumerate(stream)
                   if all(mn[a] <= p[a] < mn[a] + s for a in range(3))]
        node = {"level": level, "min": mn, "log2size": L, "ijk": (ix, iy, iz)}
        if len(members) > T and L > 0:
            node["inner"] = True
            voxels = []
            for cz in range(side_cells):
                for cy in range(side_cells):
                    for cx in range(side_cells):
                        c = (cx, cy, cz)
                        # cell c spans [mn + c*s/2^G, mn + (c+1)*s/2^G) per axis
                        inside = [g for g in members
                                  if all(c[a] * s <= (stream[g][a] - mn[a]) * side_cells
                                         < (c[a] + 1) * s for a in range(3))]
                        if inside:
                            w = min(inside)
                            centre = tuple(
                                math.floor((2 * mn[a] * side_cells + (2 * c[a] + 1) * s)
                                           / (2 * side_cells)) for a in range(3))
                            cell = cx + side_cells * (cy + side_cells * cz)
                            voxels.append((cell, centre, stream[w][3]))
            voxels.sort()
            node["voxels"] = voxels
            node["n"] = len(voxels)
            out.append(node)
            for oz in range(2):
                for oy in range(2):
                    for ox in range(2):
                        visit(level + 1, 2 * ix + ox, 2 * iy + oy, 2 * iz + oz)
        else:
            node["inner"] = False
            node["points"] = sorted(members)
            node["n"] = len(members)
            out.append(node)
        node["n_chunks"] = (node["n"] + C - 1) // C

    visit(0, 0, 0, 0)
    out.sort(key=lambda d: (d["level"],) + d["ijk"])
    return out


def snapshot_to_dicts(snap, stream=None):
    """Oracle or library snapshot -> list of node dicts like brute_force()."""
    res = []
    for node, pts, vox in snap.node_slices():
        d = {"level": int(node["level"]), "min": tuple(int(v) for v in node["min"]),
             "log2size": int(node["log2size"]), "inner": bool(node["is_inner"]),
             "n_chunks": int(node["n_chunks"])}
        if d["inner"]:
            d["voxels"] = [(int(v["cell"]), (int(v["x"]), int(v["y"]), int(v["z"])), int(v["rgba"]))
                           for v in vox]
            d["n"] = len(vox)
            assert len(pts) == 0
        else:
            d["points"] = [int(g) for g in pts["gidx"]]
            d["n"] = len(pts)
            assert len(vox) == 0
            if stream is not None:
                for p in pts:
                    g = int(p["gidx"])
                    assert (int(p["x"]), int(p["y"]), int(p["z"]), int(p["rgba"])) == stream[g]
        res.append(d)
    return res


def compare_to_brute(snap, stream, root_min, root_log2, T, C, G):
    want = brute_force(stream, root_min, root_log2, T, C, G)
    got = snapshot_to_dicts(snap, stream)
    assert len(got) == len(want), (len(got), len(want))
    for g, w in zip(got, want):
        for key in ("level", "min", "log2size", "inner", "n_chunks"):
            assert g[key] == w[key], (key, g, w)
        if w["inner"]:
            assert g["voxels"] == w["voxels"], (g["min"], g["voxels"], w["voxels"])
        else:
            assert g["points"] == w["points"], (g["min"], g["points"], w["points"])


# ----------------------------------------------------------------- invariants

def check_invariants(snap, stream_pts: np.ndarray, root_min, root_log2, T, C, G):
    """Invariants that hold at any size (vectorised numpy).

    I1 every arrival index stored exactly once, with its own record;
    I2 leaf sizes <= T except one-unit leaves; inner nodes hold > T points;
    I3 node cubes nest: 8 children per inner node, halves of the parent;
    I4 chunk count = ceil(n / C) per node;
    I8 leaf points inside their leaf; voxel cells inside the node grid and
       voxel positions inside their cells (centre floor).
    """
    nodes, points, voxels = snap.nodes, snap.points, snap.voxels
    n = len(stream_pts)
    # I1
    gidx = points["gidx"].astype(np.int64)
    assert len(gidx) == n
    assert np.array_equal(np.sort(gidx), np.arange(n))
    src = stream_pts[gidx]
    assert np.array_equal(points["x"], src["x"]) and np.array_equal(points["y"], src["y"])
    assert np.array_equal(points["z"], src["z"]) and np.array_equal(points["rgba"], rgba_of(src))
    # I4
    cnt = np.where(nodes["is_inner"] == 1, nodes["n_voxels"], nodes["n_points"]).astype(np.int64)
    assert np.array_equal(nodes["n_chunks"].astype(np.int64), (cnt + C - 1) // C)
    assert np.all(nodes["n_points"][nodes["is_inner"] == 1] == 0)
    assert np.all(nodes["n_voxels"][nodes["is_inner"] == 0] == 0)
    # I2
    leaf = nodes["is_inner"] == 0
    big = leaf & (nodes["n_points"] > T)
    assert np.all(nodes["log2size"][big] == 0)
    # I3 + subtree counts: index nodes by (level, ijk)
    L = nodes["log2size"].astype(np.int64)
    mins = nodes["min"].astype(np.int64)
    ijk = (mins - np.asarray(root_min, np.int64)) >> L[:, None]
    assert np.all(nodes["level"].astype(np.int64) + L == root_log2)
    assert np.all((ijk << L[:, None]) + np.asarray(root_min) == mins)
    key = {(int(l), int(a), int(b), int(c)): k
           for k, (l, (a, b, c)) in enumerate(zip(nodes["level"], ijk))}
    assert key.get((0, 0, 0, 0)) == 0
    for k in np.nonzero(nodes["is_inner"] == 1)[0]:
        l, (a, b, c) = int(nodes["level"][k]), ijk[k]
        for o in range(8):
            ck = (l + 1, 2 * int(a) + (o & 1), 2 * int(b) + ((o >> 1) & 1), 2 * int(c) + (o >> 2))
            assert ck in key, ("missing child", ck)
    for k in range(1, len(nodes)):
        l, (a, b, c) = int(nodes["level"][k]), ijk[k]
        pk = (l - 1, int(a) >> 1, int(b) >> 1, int(c) >> 1)
        assert pk in key and nodes["is_inner"][key[pk]] == 1, ("orphan", l, a, b, c)
    # I8 points inside leaves
    po = np.repeat(np.arange(len(nodes)), nodes["n_points"].astype(np.int64))
    for ax, f in enumerate("xyz"):
        d = points[f].astype(np.int64) - mins[po, ax]
        assert np.all((d >= 0) & (d < (np.int64(1) << L[po])))
    # inner nodes hold more than T points of the stream (subtree point count)
    # leaf points per subtree: count points whose leaf is a descendant
    # (checked through the root: all points are in leaves below it)
    # I8 voxels: cell in range, position = floor of the cell centre
    vo = np.repeat(np.arange(len(nodes)), nodes["n_voxels"].astype(np.int64))
    cells = voxels["cell"].astype(np.int64)
    assert np.all(cells < (1 << (3 * G)))
    S = np.int64(1) << G
    c3 = [cells % S, (cells // S) % S, cells // (S * S)]
    for ax, f in enumerate("xyz"):
        want = mins[vo, ax] + (((2 * c3[ax] + 1) << L[vo]) >> (G + 1))
        assert np.array_equal(voxels[f].astype(np.int64), want)
    # voxel cells unique per node
    if len(voxels):
        comb = vo * (1 << (3 * G)) + cells
        assert len(np.unique(comb)) == len(comb)
    return True


def check_allocator(snap, stats):
    """Chunk allocator accounting at rest (I4, second half): every chunk taken
    from the data region is either in exactly one node's list or in the pool
    (a compacted node's records sit in an array instead of the chunks its
    snapshot still counts)."""
    live = int(snap.nodes["n_chunks"].astype(np.int64).sum()) - int(stats.get("compact_chunks", 0))
    assert live + int(stats["chunks_pool"]) == int(stats["chunks_bumped"]), \
        (live, stats["chunks_pool"], stats["chunks_bumped"])


def assert_snapshots_equal(a, b):
    assert np.array_equal(a.nodes, b.nodes), _first_diff(a.nodes, b.nodes)
    assert np.array_equal(a.points, b.points), _first_diff(a.points, b.points)
    assert np.array_equal(a.voxels, b.voxels), _first_diff(a.voxels, b.voxels)


def _first_diff(x, y):
    if len(x) != len(y):
        return f"length {len(x)} != {len(y)}"
    bad = np.nonzero(x != y)[0]
    return f"first difference at {bad[0]}: {x[bad[0]]} != {y[bad[0]]}" if len(bad) else "equal"
