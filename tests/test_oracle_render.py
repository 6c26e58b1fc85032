"""Pins of the CPU renderer (Section 6) against values fixed by hand and by a
second formulation of the selection rule.

* Projection, pixel and depth word of single samples, computed by hand for
  matrices whose arithmetic is exact.
* The closest sample wins a pixel whatever the arrival order.
* Selection: the oracle walks the tree top down as the paper describes it
  (hide an inner node larger than 2^G pixels and visit its children). Because
  a child's screen box lies inside its parent's, that walk selects exactly
  the nodes with: in the frustum, (leaf or not larger than 2^G), and parent
  larger than 2^G (or root) -- a per-node rule, restated here in numpy with
  the same float32 operation order, and the one the GPU evaluates in
  parallel. The framebuffer equals a numpy minimum over the selected nodes'
  samples.
"""
import struct

import numpy as np
import pytest

import oracle
from helpers import points_array
from paper_2310_03567_gb300 import synth

F32 = np.float32


def bits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def ortho(world_w, world_h):
    """x, y in [0, world) -> ndc [-1, 1); w = 1 (exact when world is a power of 2)."""
    m = np.zeros(16, F32)
    m[0] = 2.0 / world_w
    m[3] = -1.0
    m[5] = 2.0 / world_h
    m[7] = -1.0
    m[15] = 1.0
    return m


def look_at_perspective(eye, target, fov_deg, aspect):
    """Row-major view-projection (float64 math, stored as float32)."""
    eye, target = np.asarray(eye, float), np.asarray(target, float)
    f = target - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0]) if abs(f[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fov_deg) / 2)
    proj = np.zeros((4, 4))
    proj[0, 0], proj[1, 1] = t / aspect, t
    proj[2, 2], proj[2, 3] = -1.0, -1.0
    proj[3, 2] = -1.0
    return (proj @ view).astype(F32).reshape(16)


def tree_of(rows, root_log2=10, T=2, G=2):
    cfg = oracle.Config.make(root_log2=root_log2, leaf_capacity=T, chunk_points=4, grid_log2=G)
    return cfg, oracle.static_build(cfg, points_array(rows))


def test_single_point_pixel_and_depth_word():
    cfg, snap = tree_of([(512, 256, 7, 10, 20, 30, 40)])
    fb, drawn, nd = oracle.render(cfg, snap, ortho(1024, 1024), 8, 4)
    # x: (512 / 512 - 1) * .5 + .5 = .5 -> 4.0 of 8; y: (256 / 512 - 1) = -.5 -> .25 -> 1.0 of 4
    want = np.full((4, 8), ~np.uint64(0), np.uint64)
    want[1, 4] = (bits(1.0) << 32) | (10 | 20 << 8 | 30 << 16 | 40 << 24)
    assert np.array_equal(fb, want)
    assert nd == 1 and drawn.tolist() == [True]


def test_points_outside_the_screen_or_behind_are_dropped():
    rows = [(1023, 0, 0, 1, 1, 1, 1), (0, 1023, 0, 2, 2, 2, 2)]
    cfg, snap = tree_of(rows, T=8)
    m = ortho(1024, 1024)
    fb, _, _ = oracle.render(cfg, snap, m, 4, 4)
    # 1023/512 - 1 = .998 -> screen 3.996 -> pixel 3; 0 -> pixel 0
    assert fb[0, 3] >> np.uint64(32) == bits(1.0) and fb[3, 0] >> np.uint64(32) == bits(1.0)
    m_shift = m.copy()
    m_shift[3] = 0.0  # x in [0, 1024) -> ndc [0, 2): right half and beyond
    fb, _, _ = oracle.render(cfg, snap, m_shift, 4, 4)
    assert int((fb != ~np.uint64(0)).sum()) == 1  # x = 1023 -> ndc 1.998: off screen
    m_back = m.copy()
    m_back[15] = -1.0  # w = -1: every sample behind the eye
    fb, drawn, _ = oracle.render(cfg, snap, m_back, 4, 4)
    assert np.all(fb == ~np.uint64(0)) and not drawn.any()


@pytest.mark.parametrize("order", [0, 1])
def test_closest_sample_wins_in_any_order(order):
    # w row picks z: both points project to ndc (0.5, 0.5) at different depths
    m = np.zeros(16, F32)
    m[0], m[5], m[15] = 1.0, 1.0, 0.0
    m[14] = 1.0  # w = z
    near, far = (64, 64, 128, 9, 9, 9, 9), (128, 128, 256, 1, 1, 1, 1)
    rows = [near, far] if order == 0 else [far, near]
    cfg, snap = tree_of(rows, T=8)
    fb, _, _ = oracle.render(cfg, snap, m, 4, 4)
    got = fb[fb != ~np.uint64(0)]
    assert len(got) == 1 and int(got[0]) == (bits(128.0) << 32) | 0x09090909


def cube_view_np(m, mins, L, W, H):
    """Per-node frustum test and size on screen (float32, same operation order)."""
    m = m.astype(F32)
    n = len(mins)
    corners = np.empty((n, 8, 3), F32)
    for k in range(8):
        for a in range(3):
            corners[:, k, a] = (mins[:, a].astype(np.int64) +
                                (np.int64((k >> a) & 1) << L.astype(np.int64))).astype(F32)
    x, y, z = corners[..., 0], corners[..., 1], corners[..., 2]
    cx = ((m[0] * x + m[1] * y) + m[2] * z) + m[3]
    cy = ((m[4] * x + m[5] * y) + m[6] * z) + m[7]
    cw = ((m[12] * x + m[13] * y) + m[14] * z) + m[15]
    front = cw > F32(0)
    culled = (np.all(cx < -cw, 1) | np.all(cx > cw, 1) | np.all(cy < -cw, 1) |
              np.all(cy > cw, 1) | np.all(~front, 1))
    with np.errstate(divide="ignore", invalid="ignore"):
        sx = ((cx / cw) * F32(0.5) + F32(0.5)) * F32(W)
        sy = ((cy / cw) * F32(0.5) + F32(0.5)) * F32(H)
    sx_lo = np.where(front, sx, np.inf).min(1)
    sx_hi = np.where(front, sx, -np.inf).max(1)
    sy_lo = np.where(front, sy, np.inf).min(1)
    sy_hi = np.where(front, sy, -np.inf).max(1)
    size = np.maximum((sx_hi - sx_lo).astype(F32), (sy_hi - sy_lo).astype(F32))
    size = np.where(np.all(front, 1), size, np.inf).astype(F32)
    return culled, size


def select_np(snap, root_min, m, W, H, G):
    nodes = snap.nodes
    L = nodes["log2size"].astype(np.int64)
    mins = nodes["min"].astype(np.int64)
    culled, size = cube_view_np(m, mins, L, W, H)
    pmin = np.asarray(root_min, np.int64) + (((mins - np.asarray(root_min, np.int64)) >> (L + 1)[:, None])
                                             << (L + 1)[:, None])
    _, psize = cube_view_np(m, pmin, L + 1, W, H)
    lod = F32(1 << G)
    root = nodes["level"] == 0
    return ~culled & ((nodes["is_inner"] == 0) | ~(size > lod)) & (root | (psize > lod))


def splat_np(m, recs, W, H):
    m = m.astype(F32)
    x, y, z = (recs[f].astype(F32) for f in "xyz")
    cx = ((m[0] * x + m[1] * y) + m[2] * z) + m[3]
    cy = ((m[4] * x + m[5] * y) + m[6] * z) + m[7]
    cw = ((m[12] * x + m[13] * y) + m[14] * z) + m[15]
    with np.errstate(divide="ignore", invalid="ignore"):
        sx = ((cx / cw) * F32(0.5) + F32(0.5)) * F32(W)
        sy = ((cy / cw) * F32(0.5) + F32(0.5)) * F32(H)
        ok = (cw > 0) & (sx >= 0) & (sx < F32(W)) & (sy >= 0) & (sy < F32(H))
    px, py = sx[ok].astype(np.int64), sy[ok].astype(np.int64)
    key = (cw[ok].view(np.uint32).astype(np.uint64) << np.uint64(32)) | recs["rgba"][ok].astype(np.uint64)
    fb = np.full(W * H, ~np.uint64(0), np.uint64)
    np.minimum.at(fb, py * W + px, key)
    return fb.reshape(H, W)


# cameras over a 2^20 mm (1 km) cube, in mm
CAMS = [
    ((-230e3, -180e3, 150e3), (524e3, 524e3, 25e3), 60.0),
    ((524e3, 524e3, 2.3e6), (524e3, 524e3, 0.0), 50.0),
    ((77e3, 128e3, 31e3), (230e3, 384e3, 10e3), 75.0),
    ((1.28e6, 1.28e6, 768e3), (1.0e6, 768e3, 0.0), 40.0),
    ((524e3, 524e3, 77e3), (524e3, 1.5e6, 77e3), 90.0),  # inside, looking along +y
]


@pytest.mark.parametrize("cam", range(len(CAMS)))
def test_selection_and_framebuffer_match_per_node_rule(cam):
    G = 4
    pts = np.concatenate([
        synth.terrain(7, 150_000, extent_m=1000.0, row_len=1000, root_log2=20),
        synth.clustered(5, 40, 60_000, root_log2=20, lo=(50.0, 50.0, 10.0),
                        hi=(1000.0, 1000.0, 200.0))])
    cfg = oracle.Config.make(root_log2=20, leaf_capacity=500, chunk_points=64, grid_log2=G)
    snap = oracle.static_build(cfg, pts)
    W, H = 320, 200
    eye, tgt, fov = CAMS[cam]
    m = look_at_perspective(eye, tgt, fov, W / H)
    fb, drawn, nd = oracle.render(cfg, snap, m, W, H)
    want = select_np(snap, (0, 0, 0), m, W, H, G)
    assert np.array_equal(drawn, want), (np.nonzero(drawn != want)[0][:5])
    assert nd == int(want.sum())
    # framebuffer: minimum over the selected nodes' samples
    sel_pts = np.repeat(drawn, snap.nodes["n_points"].astype(np.int64))
    sel_vox = np.repeat(drawn, snap.nodes["n_voxels"].astype(np.int64))
    recs = np.concatenate([snap.points[sel_pts][["x", "y", "z", "rgba"]],
                           snap.voxels[sel_vox][["x", "y", "z", "rgba"]]])
    assert np.array_equal(fb, splat_np(m, recs, W, H))


def test_far_camera_draws_only_the_root_and_near_camera_draws_leaves():
    G = 4
    pts = synth.uniform(9, 1 << 12, 20_000)
    cfg = oracle.Config.make(root_log2=12, leaf_capacity=300, chunk_points=64, grid_log2=G)
    snap = oracle.static_build(cfg, pts)
    assert snap.nodes["is_inner"][0] == 1
    far = look_at_perspective((2048.0, 2048.0, 4.0e6), (2048.0, 2048.0, 2048.0), 30.0, 1.0)
    _, drawn, nd = oracle.render(cfg, snap, far, 64, 64)
    assert nd == 1 and drawn[0]  # the root is smaller than 16 pixels: its voxels stand in
    near = look_at_perspective((2048.0, 2048.0, 9000.0), (2048.0, 2048.0, 2048.0), 60.0, 1.0)
    _, drawn, _ = oracle.render(cfg, snap, near, 1024, 1024)
    assert not drawn[0] and drawn[snap.nodes["is_inner"] == 0].any()


def test_lod_threshold_is_the_grid_resolution():
    # one inner root whose screen size lies between 2^2 and 2^4 pixels
    pts = synth.uniform(3, 1 << 10, 2_000)
    m = ortho(1 << 10, 1 << 10)  # the root spans the whole 12 x 12 screen
    for G, root_drawn in ((4, True), (2, False)):
        cfg = oracle.Config.make(root_log2=10, leaf_capacity=100, chunk_points=16, grid_log2=G)
        snap = oracle.static_build(cfg, pts)
        _, drawn, _ = oracle.render(cfg, snap, m, 12, 12)
        assert bool(drawn[0]) == root_drawn
