"""GPU renderer (Section 6) against the CPU renderer, bit for bit: the octree
built on the GPU is drawn with simlod_render, the oracle's octree of the same
stream with oracle.render, for several cameras and grid resolutions; the
frames, and the number of drawn nodes, must be identical."""
import numpy as np
import pytest

import oracle
from paper_2310_03567_gb300 import simlod, synth
from test_oracle_render import CAMS, look_at_perspective

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def scene():
    return np.concatenate([
        synth.terrain(7, 400_000, extent_m=1000.0, row_len=1000, root_log2=20),
        synth.clustered(5, 60, 200_000, root_log2=20, lo=(50.0, 50.0, 10.0),
                        hi=(1000.0, 1000.0, 200.0))])


def gpu_tree(pts, **kw):
    cfg = simlod.default_config(root_log2=20, max_batch_points=1 << 18, spill_capacity=1 << 21,
                                backlog_capacity=1 << 21, max_nodes=1 << 18, **kw)
    arena = simlod.make_arena(cfg, 1 << 30)
    t = simlod.Octree(cfg, arena, stream=torch.cuda.Stream())
    ts = [simlod.points_tensor(pts[k:k + (1 << 18)]) for k in range(0, len(pts), 1 << 18)]
    t.insert_many(ts)
    assert t.sync() == simlod.OK
    return t


def gpu_frame(tree, m, W, H, clear=True, fb=None):
    if fb is None:
        fb = torch.empty((H, W), dtype=torch.int64, device="cuda")
    tree.render(m, fb, clear=clear)
    assert tree.sync() == simlod.OK
    return fb, fb.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("G,T", [(4, 500), (7, 5000)])
def test_frames_match_the_oracle(G, T):
    pts = scene()
    tree = gpu_tree(pts, leaf_capacity=T, chunk_points=64 if G == 4 else 1000, grid_log2=G)
    cfg = oracle.Config.make(root_log2=20, leaf_capacity=T,
                             chunk_points=64 if G == 4 else 1000, grid_log2=G)
    snap = oracle.static_build(cfg, pts)
    W, H = 480, 270
    for eye, tgt, fov in CAMS:
        m = look_at_perspective(eye, tgt, fov, W / H)
        _, got = gpu_frame(tree, m, W, H)
        want, drawn, nd = oracle.render(cfg, snap, m, W, H)
        assert np.array_equal(got, want), int((got != want).sum())
        st = tree.stats()
        assert st["render_nodes"] == nd
        expect = int(np.where(snap.nodes["is_inner"] == 1, snap.nodes["n_voxels"],
                              snap.nodes["n_points"])[drawn].sum())
        assert st["render_samples"] == expect


def test_two_octrees_share_one_frame():
    pts = scene()
    a = gpu_tree(pts[: len(pts) // 2], leaf_capacity=2000, grid_log2=6)
    b = gpu_tree(pts[len(pts) // 2:], leaf_capacity=2000, grid_log2=6)
    W, H = 320, 180
    m = look_at_perspective(*CAMS[0][:2], CAMS[0][2], W / H)
    _, fa = gpu_frame(a, m, W, H)
    _, fb_ = gpu_frame(b, m, W, H)
    buf, _ = gpu_frame(a, m, W, H)
    b.stream.wait_stream(a.stream)
    _, both = gpu_frame(b, m, W, H, clear=False, fb=buf)
    assert np.array_equal(both, np.minimum(fa, fb_))


def test_render_follows_inserts_on_the_stream():
    pts = scene()
    half = len(pts) // 2
    cfg = simlod.default_config(root_log2=20, leaf_capacity=3000, grid_log2=5,
                                max_batch_points=1 << 20, spill_capacity=1 << 21,
                                backlog_capacity=1 << 21, max_nodes=1 << 18)
    tree = simlod.Octree(cfg, simlod.make_arena(cfg, 1 << 30), stream=torch.cuda.Stream())
    W, H = 256, 256
    m = look_at_perspective(*CAMS[1][:2], CAMS[1][2], 1.0)
    fb0 = torch.empty((H, W), dtype=torch.int64, device="cuda")
    fb1 = torch.empty((H, W), dtype=torch.int64, device="cuda")
    tree.insert(simlod.points_tensor(pts[:half]), check=False)
    tree.render(m, fb0)  # enqueued after the first insert, before the second
    tree.insert(simlod.points_tensor(pts[half:]), check=False)
    tree.render(m, fb1)
    assert tree.sync() == simlod.OK
    ocfg = oracle.Config.make(root_log2=20, leaf_capacity=3000, grid_log2=5)
    for fb, n in ((fb0, half), (fb1, len(pts))):
        want, _, _ = oracle.render(ocfg, oracle.static_build(ocfg, pts[:n]), m, W, H)
        assert np.array_equal(fb.cpu().numpy().view(np.uint64), want)


def test_render_rejects_bad_arguments():
    tree = gpu_tree(scene()[:1000], leaf_capacity=100, grid_log2=4)
    m = np.eye(4, dtype=np.float32).reshape(16)
    lib = simlod.load()
    fb = torch.empty((4, 4), dtype=torch.int64, device="cuda")
    assert lib.simlod_render(tree._h, m.ctypes.data, 0, 4, fb.data_ptr(), 1, None) == \
        simlod.ERR_INVALID_ARG
    assert lib.simlod_render(tree._h, m.ctypes.data, 4, 4, fb.data_ptr() + 4, 1, None) == \
        simlod.ERR_INVALID_ARG
    assert lib.simlod_render(tree._h, None, 4, 4, fb.data_ptr(), 1, None) == simlod.ERR_INVALID_ARG
