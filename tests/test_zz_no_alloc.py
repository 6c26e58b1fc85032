"""The no-allocation entry point gives the oracle's voxels and allocates nothing.

simlod_sample_node_noalloc is meant for callers that cannot allocate device
memory when they need voxel sampling (a running frame loop, or code that lives
inside another framework's memory management): its scratch is a fixed device
array in the library instead of a caller arena. Here it is called through the
C ABI twice in a row, with different batches. Each result must equal the root
voxels of the oracle's closed-form octree of the same points (oracle/static.c)
and those of the regular insert path (simlod_insert_batch into a fresh octree
whose root splits). Voxels are integers, so the comparisons are exact. A
further call must leave the device's free memory and torch's allocated bytes
unchanged.

This file sorts last on purpose, so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _root_voxels_by_oracle(pts: np.ndarray) -> np.ndarray:
    cfg = oracle.Config.make(root_log2=L, leaf_capacity=1000, grid_log2=G)
    snap = oracle.static_build(cfg, pts)
    root = snap.nodes[0]
    assert root["level"] == 0 and root["is_inner"] == 1
    out = snap.voxels[:int(root["n_voxels"])]  # the root's voxels come first
    # the oracle's voxel records have the same fields and layout
    assert out.dtype.names == simlod.VOXEL_REC_DTYPE.names
    return out.view(simlod.VOXEL_REC_DTYPE)


def test_noalloc_matches_oracle_and_insert_path_twice():
    stream = torch.cuda.Stream()
    # call 1: points spread over the whole cube (mostly one point per cell)
    a = synth.uniform(101, 1 << L, 100_000)
    # call 2: the largest accepted batch packed into a 2^11 cube (about 5^3
    # cells of 512 units), so that many points from many warps contend for
    # each cell and stale table entries from call 1 would show up
    b = synth.uniform(102, 1 << 11, simlod_max())
    b["x"] += 20_000
    b["y"] += 3_000
    b["z"] += 41_000
    got_a = _noalloc(a, stream)
    got_b = _noalloc(b, stream)
    for got, pts in ((got_a, a), (got_b, b)):
        want = _root_voxels_by_oracle(pts)
        assert len(got) == len(want) and np.array_equal(got, want)
        by_insert = _root_voxels_by_insert(pts)
        assert len(got) == len(by_insert) and np.array_equal(got, by_insert)


def test_noalloc_allocates_nothing():
    lib = simlod.load()
    stream = torch.cuda.Stream()
    pts = synth.uniform(103, 1 << L, 50_000)
    d_pts = simlod.points_tensor(pts)
    d_out = torch.empty((len(pts), simlod.VOXEL_REC_DTYPE.itemsize), dtype=torch.uint8,
                        device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())

    def call():
        rc = lib.simlod_sample_node_noalloc(d_pts.data_ptr(), len(pts),
                                            (ctypes.c_int32 * 3)(0, 0, 0), L, G,
                                            d_out.data_ptr(), len(pts), d_cnt.data_ptr(),
                                            stream.cuda_stream)
        assert rc == simlod.OK, simlod.status_string(rc)
        stream.synchronize()

    call()  # warm-up: the first call in the context loads the device code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    assert 0 < int(d_cnt.item()) <= len(pts)


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = simlod.load()
    d_out = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = lib.simlod_sample_node_noalloc(d_out.data_ptr(), simlod_max() + 1,
                                        (ctypes.c_int32 * 3)(0, 0, 0), L, G, d_out.data_ptr(),
                                        1 << 30, d_out.data_ptr(), None)
    assert rc == simlod.ERR_INVALID_ARG


def simlod_max() -> int:
    return 131072  # SIMLOD_NOALLOC_MAX_POINTS in include/simlod.h
