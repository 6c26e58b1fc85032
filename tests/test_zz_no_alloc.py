"""The no-allocation entry point gives the same voxels as the arena path.

simlod_sample_node_noalloc is meant for callers that cannot allocate device
memory when they need voxel sampling (a running frame loop, or code that lives
inside another framework's memory management): its scratch is a fixed device
array in the library instead of a caller arena. Here it is called through the
C ABI twice in a row, with different batches, and each result must equal the
root voxels that the regular insert path (simlod_insert_batch into a fresh
octree whose root splits) produces for the same points. Voxels are integers,
so the comparison is exact.

This file sorts last on purpose, so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2310_03567_gb300 import simlod, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L, G = 16, 7  # a 2^16 cube sampled on the paper's 128^3 grid


def _noalloc(pts: np.ndarray, stream) -> np.ndarray:
    lib = simlod.load()
    n = len(pts)
    d_pts = simlod.points_tensor(pts)
    d_out = torch.empty((max(n, 1), simlod.VOXEL_REC_DTYPE.itemsize), dtype=torch.uint8,
                        device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    rc = lib.simlod_sample_node_noalloc(d_pts.data_ptr(), n, (ctypes.c_int32 * 3)(0, 0, 0), L, G,
                                        d_out.data_ptr(), max(n, 1), d_cnt.data_ptr(),
                                        stream.cuda_stream)
    assert rc == simlod.OK, simlod.status_string(rc)
    stream.synchronize()
    k = int(d_cnt.item())
    assert 0 < k <= n
    recs = d_out[:k].cpu().numpy().copy().view(simlod.VOXEL_REC_DTYPE).reshape(-1)
    return np.sort(recs, order="cell")


def _root_voxels_by_insert(pts: np.ndarray) -> np.ndarray:
    cfg = simlod.default_config(root_log2=L, leaf_capacity=1000, grid_log2=G,
                                max_batch_points=1 << 18, spill_capacity=1 << 18,
                                backlog_capacity=1 << 20, max_nodes=1 << 16)
    tree = simlod.Octree(cfg, simlod.make_arena(cfg, 1 << 29), stream=torch.cuda.Stream())
    tree.insert(simlod.points_tensor(pts))
    snap = tree.snapshot()
    root = snap.nodes[0]
    assert root["level"] == 0 and root["is_inner"] == 1
    out = snap.voxels[:int(root["n_voxels"])].copy()  # the root's voxels come first
    tree.close()
    return out


def test_noalloc_matches_insert_path_twice():
    stream = torch.cuda.Stream()
    # call 1: points spread over the whole cube (mostly one point per cell)
    a = synth.uniform(101, 1 << L, 100_000)
    # call 2: the largest accepted batch packed into 4^3 cells, so that many
    # points from many warps contend for each cell and stale table entries
    # from call 1 would show up
    b = synth.uniform(102, 1 << 11, simlod_max())
    b["x"] += 20_000
    b["y"] += 3_000
    b["z"] += 41_000
    got_a = _noalloc(a, stream)
    got_b = _noalloc(b, stream)
    want_a = _root_voxels_by_insert(a)
    want_b = _root_voxels_by_insert(b)
    assert len(got_a) == len(want_a) and np.array_equal(got_a, want_a)
    assert len(got_b) == len(want_b) and np.array_equal(got_b, want_b)


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = simlod.load()
    d_out = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = lib.simlod_sample_node_noalloc(d_out.data_ptr(), simlod_max() + 1,
                                        (ctypes.c_int32 * 3)(0, 0, 0), L, G, d_out.data_ptr(),
                                        1 << 30, d_out.data_ptr(), None)
    assert rc == simlod.ERR_INVALID_ARG


def simlod_max() -> int:
    return 131072  # SIMLOD_NOALLOC_MAX_POINTS in include/simlod.h
