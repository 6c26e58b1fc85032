"""ctypes binding of ``libsimlod.so`` (the C ABI in ``include/simlod.h``).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels. PyTorch provides the device arena (a uint8 CUDA tensor the
caller owns, like the paper's persistent buffer, Section 3.2) and streams.
There is no CPU fallback: if the library cannot be loaded, importing the
binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB_PATH

OK = 0
ERR_INVALID_ARG = -1
ERR_OUT_OF_BOUNDS = -2
ERR_ARENA_FULL = -3
ERR_BACKLOG_FULL = -4
ERR_SPILL_FULL = -5
ERR_ITER_CAP = -6
ERR_TIMEOUT = -7
ERR_POISONED = -8
ERR_CUDA = -9
ERR_NODES_FULL = -10
ERR_TOO_MANY_POINTS = -11

N_KERNELS = 8


class SimlodError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("root_min", ctypes.c_int32 * 3), ("root_log2", ctypes.c_uint32),
                ("leaf_capacity", ctypes.c_uint32), ("chunk_points", ctypes.c_uint32),
                ("grid_log2", ctypes.c_uint32), ("max_expand_iters", ctypes.c_uint32),
                ("max_batch_points", ctypes.c_uint64), ("spill_capacity", ctypes.c_uint64),
                ("backlog_capacity", ctypes.c_uint64), ("max_nodes", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class NodeRec(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("is_inner", ctypes.c_uint32),
                ("min", ctypes.c_int32 * 3), ("log2size", ctypes.c_uint32),
                ("n_points", ctypes.c_uint64), ("n_voxels", ctypes.c_uint64),
                ("n_chunks", ctypes.c_uint64)]


class Snapshot_t(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("nodes_capacity", ctypes.c_uint64),
                ("points", ctypes.c_void_p), ("points_capacity", ctypes.c_uint64),
                ("voxels", ctypes.c_void_p), ("voxels_capacity", ctypes.c_uint64),
                ("n_nodes", ctypes.c_uint64), ("n_points", ctypes.c_uint64),
                ("n_voxels", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "batches", "points", "rejected_batches", "spilled", "splits", "voxels",
        "iterations_max", "rounds", "nodes", "chunks_bumped", "chunks_pool", "arena_bytes", "data_bytes",
        "data_used", "last_points", "last_spilled", "last_splits", "last_voxels",
        "last_iterations")] + [("sticky_status", ctypes.c_int32),
                               ("device_error_bits", ctypes.c_uint32),
                               ("render_nodes", ctypes.c_uint64),
                               ("render_samples", ctypes.c_uint64),
                               ("compact_nodes", ctypes.c_uint64),
                               ("compact_chunks", ctypes.c_uint64),
                               ("compacted_total", ctypes.c_uint64),
                               ("compact_chunks_freed", ctypes.c_uint64),
                               ("decompacted_total", ctypes.c_uint64)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


N_PHASES = 8


class Timing(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p * N_KERNELS), ("launches", ctypes.c_uint64 * N_KERNELS),
                ("ms", ctypes.c_double * N_KERNELS),
                ("phase_name", ctypes.c_char_p * N_PHASES),
                ("phase_ms", ctypes.c_double * N_PHASES)]


# numpy views of the snapshot records (same layout as the C structs)
NODE_DTYPE = np.dtype([("level", "<u4"), ("is_inner", "<u4"), ("min", "<i4", (3,)),
                       ("log2size", "<u4"), ("n_points", "<u8"), ("n_voxels", "<u8"),
                       ("n_chunks", "<u8")])
POINT_REC_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("rgba", "<u4"),
                            ("gidx", "<u4")])
VOXEL_REC_DTYPE = np.dtype([("cell", "<u4"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                            ("rgba", "<u4")])

_lib = None

# (name, restype, argtypes) of every exported function
_P, _U64, _I32, _U32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
SIGNATURES = {
    "simlod_config_default": (None, [ctypes.POINTER(Config)]),
    "simlod_arena_bytes": (_I32, [ctypes.POINTER(Config), _U64, ctypes.POINTER(_U64)]),
    "simlod_create": (_I32, [ctypes.POINTER(Config), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "simlod_insert_batch": (_I32, [_P, _P, _U64, _P]),
    "simlod_insert_batch_host": (_I32, [_P, _P, _U64, _P]),
    "simlod_insert_batches": (_I32, [_P, _P, _P, _U32, _P]),
    "simlod_insert_batches_host": (_I32, [_P, _P, _P, _U32, _P, _P, _P, _P]),
    "simlod_frame_update": (_I32, [_P, _P, _P, _U32, _U64, _P, ctypes.POINTER(_U32)]),
    "simlod_reset": (_I32, [_P, _P]),
    "simlod_sync": (_I32, [_P]),
    "simlod_get_stats": (_I32, [_P, ctypes.POINTER(Stats)]),
    "simlod_snapshot": (_I32, [_P, ctypes.POINTER(Snapshot_t)]),
    "simlod_set_timing": (_I32, [_P, _I32, _I32]),
    "simlod_get_timing": (_I32, [_P, ctypes.POINTER(Timing)]),
    "simlod_destroy": (_I32, [_P]),
    "simlod_status_string": (ctypes.c_char_p, [_I32]),
    "simlod_sample_node_noalloc": (_I32, [_P, _U64, ctypes.POINTER(ctypes.c_int32), _U32, _U32,
                                          _P, _U64, _P, _P]),
    "simlod_render": (_I32, [_P, _P, _U32, _U32, _P, _I32, _P]),
    "simlod_set_launch_width": (_I32, [_P, _U32, ctypes.POINTER(_U32)]),
    "simlod_set_wait_limits": (_I32, [_P, _U64, _U64]),
    "simlod_restore": (_I32, [_P, ctypes.POINTER(Snapshot_t), _P]),
    "simlod_plan_create": (_I32, [_P, _P, _P, _U32, _P, ctypes.POINTER(_P)]),
    "simlod_plan_run": (_I32, [_P, _P]),
    "simlod_plan_info": (_I32, [_P, _P, ctypes.POINTER(_U32)]),
    "simlod_plan_destroy": (_I32, [_P]),
    "simlod_plan_autotune": (_I32, [_P, _P, _P, _U32, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "simlod_variant_info": (_I32, [_U32, _P]),
    "simlod_compact": (_I32, [_P, _U32, _P]),
    "simlod_progress": (_I32, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "simlod_insert_batches_budget": (_I32, [_P, _P, _P, _U32, _U64, _P]),
}


class PlanParams(ctypes.Structure):
    _fields_ = [("merge_points", ctypes.c_uint64), ("blocks_per_sm", ctypes.c_uint32),
                ("use_graph", ctypes.c_uint32), ("variant", ctypes.c_uint32)]

    def as_dict(self):
        return {"merge_points": int(self.merge_points), "blocks_per_sm": int(self.blocks_per_sm),
                "use_graph": int(self.use_graph), "variant": int(self.variant)}


class VariantDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "threads_per_block", "max_blocks_per_sm", "node_cache", "store_unroll", "descent_group",
        "smem_bytes")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


N_VARIANTS = 4  # SIMLOD_N_VARIANTS


def variant_info(variant: int) -> dict:
    """Block and tile parameters of kernel instance `variant` on the current
    device (simlod_variant_info)."""
    d = VariantDesc()
    rc = load().simlod_variant_info(variant, ctypes.byref(d))
    if rc != OK:
        raise SimlodError(rc, "simlod_variant_info")
    return d.as_dict()


def load(path: str | None = None):
    """Load (building first if needed) the CUDA library; raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = LIB_PATH
        if not os.path.exists(path):
            _build.build_library()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().simlod_status_string(status).decode()
    except Exception:
        return f"status {status}"


def view_proj(eye, target, fov_deg: float, aspect: float, up=(0.0, 0.0, 1.0)):
    """Row-major 4x4 view-projection (16 float32) for simlod_render: a camera
    at `eye` looking at `target` (coordinates in the octree's integer units),
    vertical field of view fov_deg; depth = clip w = distance along the view
    direction."""
    import numpy as _np
    eye, target = _np.asarray(eye, float), _np.asarray(target, float)
    f = target - eye
    f /= _np.linalg.norm(f)
    u0 = _np.asarray(up, float)
    if abs(float(f @ u0)) > 0.99:
        u0 = _np.array([0.0, 1.0, 0.0])
    s_ = _np.cross(f, u0)
    s_ /= _np.linalg.norm(s_)
    u = _np.cross(s_, f)
    view = _np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s_, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / _np.tan(_np.radians(fov_deg) / 2)
    proj = _np.zeros((4, 4))
    proj[0, 0], proj[1, 1] = t / aspect, t
    proj[2, 2], proj[2, 3], proj[3, 2] = -1.0, -1.0, -1.0
    return (proj @ view).astype(_np.float32).reshape(16)


def default_config(**overrides) -> Config:
    cfg = Config()
    load().simlod_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "root_min":
            for a in range(3):
                cfg.root_min[a] = int(v[a])
        else:
            setattr(cfg, k, int(v))
    return cfg


def arena_bytes(cfg: Config, data_bytes: int) -> int:
    out = ctypes.c_uint64()
    rc = load().simlod_arena_bytes(ctypes.byref(cfg), data_bytes, ctypes.byref(out))
    if rc != OK:
        raise SimlodError(rc, "simlod_arena_bytes")
    return int(out.value)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Snapshot:
    """Canonical octree (numpy structured arrays, same fields as the oracle)."""

    def __init__(self, nodes, points, voxels):
        self.nodes, self.points, self.voxels = nodes, points, voxels

    def node_slices(self):
        po = np.concatenate([[0], np.cumsum(self.nodes["n_points"])]).astype(np.int64)
        vo = np.concatenate([[0], np.cumsum(self.nodes["n_voxels"])]).astype(np.int64)
        for k in range(len(self.nodes)):
            yield (self.nodes[k], self.points[po[k]:po[k + 1]], self.voxels[vo[k]:vo[k + 1]])


class Octree:
    """One octree in a caller-owned device arena.

    ``arena`` is a uint8 CUDA tensor (or an int device pointer with
    ``arena_nbytes``); it must outlive the octree.
    """

    def __init__(self, cfg: Config, arena, stream=None, arena_nbytes: int | None = None):
        self._lib = load()
        self.cfg = cfg
        self.arena = arena  # keep the tensor alive
        if isinstance(arena, int):
            ptr, nbytes = arena, int(arena_nbytes)
        else:
            ptr, nbytes = arena.data_ptr(), arena.numel() * arena.element_size()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.simlod_create(ctypes.byref(cfg), ptr, nbytes, _stream_ptr(stream),
                                     ctypes.byref(h))
        if rc != OK:
            raise SimlodError(rc, "simlod_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def _order(self, stream, tensor=None):
        """Make `stream` wait for the caller's current stream (which produced
        the batch) and keep `tensor` from being recycled before `stream` has
        read it."""
        s = stream if stream is not None else self.stream
        if s is None or isinstance(s, int):
            return s
        import torch
        cur = torch.cuda.current_stream()
        if cur.cuda_stream != s.cuda_stream:
            s.wait_stream(cur)
            if tensor is not None:
                tensor.record_stream(s)
        return s

    def insert(self, pts, stream=None, check: bool = True) -> int:
        """Insert a batch from a CUDA tensor of 16-byte records (uint8 [n,16],
        int32 [n,4] or any contiguous tensor of n*16 bytes)."""
        nbytes = pts.numel() * pts.element_size()
        if nbytes % 16:
            raise ValueError("points must be 16-byte records")
        s = self._order(stream, pts)
        rc = self._lib.simlod_insert_batch(self._h, pts.data_ptr(), nbytes // 16, _stream_ptr(s))
        if check and rc != OK:
            raise SimlodError(rc, "simlod_insert_batch")
        return rc

    def insert_ptr(self, ptr: int, n: int, stream=None) -> int:
        return self._lib.simlod_insert_batch(
            self._h, ptr, n, _stream_ptr(stream if stream is not None else self.stream))

    def insert_host(self, pts: np.ndarray, stream=None, check: bool = True) -> int:
        """Insert a batch held in host memory (numpy array of 16-byte records
        or a pinned CPU tensor)."""
        if isinstance(pts, np.ndarray):
            a = np.ascontiguousarray(pts)
            ptr, n = a.ctypes.data, a.nbytes // 16
        else:
            ptr, n = pts.data_ptr(), pts.numel() * pts.element_size() // 16
        rc = self._lib.simlod_insert_batch_host(
            self._h, ptr, n, _stream_ptr(stream if stream is not None else self.stream))
        if check and rc != OK:
            raise SimlodError(rc, "simlod_insert_batch_host")
        return rc

    def frame_update(self, batches, budget_ns: int, stream=None) -> tuple[int, int]:
        """Apply the batches (CUDA tensors) in order within a time budget;
        returns (status, batches consumed)."""
        n = len(batches)
        for b in batches:
            self._order(stream, b)
        ptrs = (ctypes.c_void_p * max(n, 1))(*[b.data_ptr() for b in batches])
        counts = (ctypes.c_uint64 * max(n, 1))(
            *[b.numel() * b.element_size() // 16 for b in batches])
        consumed = ctypes.c_uint32()
        rc = self._lib.simlod_frame_update(
            self._h, ptrs, counts, n, budget_ns,
            _stream_ptr(stream if stream is not None else self.stream), ctypes.byref(consumed))
        return rc, int(consumed.value)

    def insert_many(self, batches, stream=None, check: bool = True) -> int:
        """Fused form: one persistent launch over a list of CUDA tensors
        (asynchronous; errors and rejections surface at sync())."""
        n = len(batches)
        s = None
        for b in batches:
            s = self._order(stream, b)
        if s is None:
            s = stream if stream is not None else self.stream
        ptrs = (ctypes.c_void_p * max(n, 1))(*[b.data_ptr() for b in batches])
        counts = (ctypes.c_uint64 * max(n, 1))(
            *[b.numel() * b.element_size() // 16 for b in batches])
        rc = self._lib.simlod_insert_batches(self._h, ptrs, counts, n, _stream_ptr(s))
        if check and rc != OK:
            raise SimlodError(rc, "simlod_insert_batches")
        return rc

    def insert_many_ptrs(self, ptrs, counts, stream=None, budget_ns: int | None = None) -> int:
        """Fused form over raw device pointers (no stream ordering done here).
        With budget_ns, batches after the first start only while the launch
        has run for at most that long (simlod_insert_batches_budget); the rest
        are dropped, and progress() tells how many were applied."""
        n = len(ptrs)
        p = (ctypes.c_void_p * max(n, 1))(*ptrs)
        c = (ctypes.c_uint64 * max(n, 1))(*counts)
        s = _stream_ptr(stream if stream is not None else self.stream)
        if budget_ns is not None:
            return self._lib.simlod_insert_batches_budget(self._h, p, c, n, int(budget_ns), s)
        return self._lib.simlod_insert_batches(self._h, p, c, n, s)

    def insert_many_host(self, host_batches, dst, ready, copy_stream, stream=None,
                         check: bool = True) -> int:
        """Fused form fed from page-locked host memory: each batch (a pinned
        CPU tensor of 16-byte records) is copied into `dst` (a CUDA tensor
        with room for all of them) on copy_stream, and the persistent launch
        starts each batch once its copy has finished (flag words in `ready`,
        an int32 CUDA tensor with one word per batch). Asynchronous: the host
        batches must stay alive until the launch has passed them (dst and
        ready are kept from reuse by the caching allocator here)."""
        n = len(host_batches)
        s = self._order(stream)
        for t in (dst, ready):
            for st in (s, copy_stream):
                if st is not None and not isinstance(st, int):
                    t.record_stream(st)
        total = sum(b.numel() * b.element_size() for b in host_batches)
        if dst.numel() * dst.element_size() < total or ready.numel() < n:
            raise ValueError("dst or ready is too small")
        ptrs = (ctypes.c_void_p * max(n, 1))(*[b.data_ptr() for b in host_batches])
        counts = (ctypes.c_uint64 * max(n, 1))(
            *[b.numel() * b.element_size() // 16 for b in host_batches])
        rc = self._lib.simlod_insert_batches_host(self._h, ptrs, counts, n, dst.data_ptr(),
                                                  ready.data_ptr(), _stream_ptr(s),
                                                  _stream_ptr(copy_stream))
        if check and rc != OK:
            raise SimlodError(rc, "simlod_insert_batches_host")
        return rc

    def reset(self, stream=None):
        rc = self._lib.simlod_reset(self._h, _stream_ptr(stream if stream is not None else self.stream))
        if rc != OK:
            raise SimlodError(rc, "simlod_reset")

    def sync(self) -> int:
        return self._lib.simlod_sync(self._h)

    def stats(self) -> dict:
        st = Stats()
        rc = self._lib.simlod_get_stats(self._h, ctypes.byref(st))
        if rc != OK:
            raise SimlodError(rc, "simlod_get_stats")
        return st.as_dict()

    def set_timing(self, enable: bool, clear: bool = False):
        self._lib.simlod_set_timing(self._h, int(enable), int(clear))

    def timing(self) -> dict:
        t = Timing()
        rc = self._lib.simlod_get_timing(self._h, ctypes.byref(t))
        if rc != OK:
            raise SimlodError(rc, "simlod_get_timing")
        return {t.name[k].decode(): (int(t.launches[k]), float(t.ms[k])) for k in range(N_KERNELS)}

    def phase_times(self) -> dict:
        """Milliseconds the fused form spent per phase since the last clear."""
        t = Timing()
        rc = self._lib.simlod_get_timing(self._h, ctypes.byref(t))
        if rc != OK:
            raise SimlodError(rc, "simlod_get_timing")
        return {t.phase_name[k].decode(): float(t.phase_ms[k]) for k in range(N_PHASES)}

    def render(self, view_proj, framebuffer, clear: bool = True, stream=None) -> None:
        """Draw into framebuffer (a CUDA uint64/int64 tensor of [height, width])
        with the row-major 4x4 view_proj (16 floats); see simlod_render."""
        import numpy as _np
        m = _np.ascontiguousarray(_np.asarray(view_proj, dtype=_np.float32).reshape(16))
        if framebuffer.dim() != 2 or framebuffer.element_size() != 8 or not framebuffer.is_cuda \
                or not framebuffer.is_contiguous():
            raise ValueError("framebuffer must be a contiguous [height, width] 8-byte CUDA tensor")
        height, width = framebuffer.shape
        st = stream if stream is not None else self.stream
        self._order(st, framebuffer)
        rc = self._lib.simlod_render(self._h, m.ctypes.data, width, height,
                                     framebuffer.data_ptr(), int(clear), _stream_ptr(st))
        if rc != OK:
            raise SimlodError(rc, "simlod_render")

    def restore(self, snap, stream=None) -> None:
        """Replace the octree with a canonical snapshot (this library's or the
        oracle's: same record layout); see simlod_restore."""
        nodes = np.ascontiguousarray(snap.nodes)
        points = np.ascontiguousarray(snap.points)
        voxels = np.ascontiguousarray(snap.voxels)
        s = Snapshot_t()
        s.nodes, s.nodes_capacity = nodes.ctypes.data, len(nodes)
        s.points, s.points_capacity = points.ctypes.data if len(points) else None, len(points)
        s.voxels, s.voxels_capacity = voxels.ctypes.data if len(voxels) else None, len(voxels)
        s.n_nodes, s.n_points, s.n_voxels = len(nodes), len(points), len(voxels)
        st = stream if stream is not None else self.stream
        rc = self._lib.simlod_restore(self._h, ctypes.byref(s), _stream_ptr(st))
        if rc != OK:
            raise SimlodError(rc, "simlod_restore")

    def set_launch_width(self, blocks_per_sm: int) -> int:
        """Blocks per SM of this handle's persistent launches (0 = all that
        fit); returns the maximum that fits."""
        mx = ctypes.c_uint32()
        rc = self._lib.simlod_set_launch_width(self._h, blocks_per_sm, ctypes.byref(mx))
        if rc != OK:
            raise SimlodError(rc, "simlod_set_launch_width")
        return int(mx.value)

    def progress(self) -> tuple[int, int]:
        """(batches finished, batches submitted) of this handle's persistent
        launches; reads host memory only (simlod_progress)."""
        fin, sub = ctypes.c_uint64(), ctypes.c_uint64()
        rc = self._lib.simlod_progress(self._h, ctypes.byref(fin), ctypes.byref(sub))
        if rc != OK:
            raise SimlodError(rc, "simlod_progress")
        return int(fin.value), int(sub.value)

    def compact(self, idle_updates: int = 0, stream=None) -> None:
        """Turn the chunk lists of nodes idle for idle_updates updates into
        contiguous arrays (simlod_compact); asynchronous on the stream."""
        st = stream if stream is not None else self.stream
        rc = self._lib.simlod_compact(self._h, idle_updates, _stream_ptr(st))
        if rc != OK:
            raise SimlodError(rc, "simlod_compact")

    def set_wait_limits(self, barrier_ns: int = 0, ready_ns: int = 0) -> None:
        """Time limits of a persistent launch's grid-barrier and ready-flag
        waits (0 = the default of 2 s)."""
        rc = self._lib.simlod_set_wait_limits(self._h, barrier_ns, ready_ns)
        if rc != OK:
            raise SimlodError(rc, "simlod_set_wait_limits")

    def plan(self, ptrs, counts, merge_points: int = 0, blocks_per_sm: int = 0,
             use_graph: bool = True, variant: int = 0) -> "Plan":
        """Batched form over raw 16-byte-aligned device pointers (kept by the
        plan; the caller keeps the buffers alive and orders their writes)."""
        return Plan(self, ptrs, counts,
                    PlanParams(merge_points, blocks_per_sm, int(use_graph), variant))

    def autotune(self, ptrs, counts, stream=None):
        """Fastest batched-form parameters for this batch list (resets the
        octree); returns (PlanParams, ms)."""
        n = len(ptrs)
        p = (ctypes.c_void_p * max(n, 1))(*ptrs)
        c = (ctypes.c_uint64 * max(n, 1))(*counts)
        best = PlanParams()
        ms = ctypes.c_double()
        st = stream if stream is not None else self.stream
        rc = self._lib.simlod_plan_autotune(self._h, p, c, n, _stream_ptr(st), ctypes.byref(best),
                                            ctypes.byref(ms))
        if rc != OK:
            raise SimlodError(rc, "simlod_plan_autotune")
        return best, float(ms.value)

    def snapshot(self) -> Snapshot:
        s = Snapshot_t()
        rc = self._lib.simlod_snapshot(self._h, ctypes.byref(s))
        if rc != OK:
            raise SimlodError(rc, "simlod_snapshot (sizes)")
        nodes = np.zeros(s.n_nodes, NODE_DTYPE)
        points = np.zeros(s.n_points, POINT_REC_DTYPE)
        voxels = np.zeros(s.n_voxels, VOXEL_REC_DTYPE)
        s.nodes, s.nodes_capacity = nodes.ctypes.data, len(nodes)
        s.points, s.points_capacity = (points.ctypes.data if len(points) else None), len(points)
        s.voxels, s.voxels_capacity = (voxels.ctypes.data if len(voxels) else None), len(voxels)
        rc = self._lib.simlod_snapshot(self._h, ctypes.byref(s))
        if rc != OK:
            raise SimlodError(rc, "simlod_snapshot")
        return Snapshot(nodes, points, voxels)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.simlod_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def points_tensor(pts: np.ndarray, device="cuda"):
    """Copy 16-byte point records to a uint8 [n, 16] CUDA tensor."""
    import torch
    a = np.ascontiguousarray(pts).view(np.uint8).reshape(-1, 16)
    return torch.from_numpy(a).to(device)


def make_arena(cfg: Config, data_bytes: int, device="cuda"):
    """Allocate a uint8 CUDA tensor large enough for cfg and data_bytes."""
    import torch
    return torch.empty(arena_bytes(cfg, data_bytes), dtype=torch.uint8, device=device)


class Plan:
    """A batched-form plan bound to an Octree (see simlod_plan_create)."""

    def __init__(self, tree: "Octree", ptrs, counts, params: PlanParams):
        self.tree = tree
        n = len(ptrs)
        p = (ctypes.c_void_p * max(n, 1))(*ptrs)
        c = (ctypes.c_uint64 * max(n, 1))(*counts)
        h = ctypes.c_void_p()
        rc = tree._lib.simlod_plan_create(tree._h, p, c, n, ctypes.byref(params), ctypes.byref(h))
        if rc != OK:
            raise SimlodError(rc, "simlod_plan_create")
        self._h = h

    def run(self, stream=None) -> int:
        st = stream if stream is not None else self.tree.stream
        return self.tree._lib.simlod_plan_run(self._h, _stream_ptr(st))

    def info(self):
        p = PlanParams()
        g = ctypes.c_uint32()
        rc = self.tree._lib.simlod_plan_info(self._h, ctypes.byref(p), ctypes.byref(g))
        if rc != OK:
            raise SimlodError(rc, "simlod_plan_info")
        return p.as_dict(), bool(g.value)

    def close(self):
        if getattr(self, "_h", None):
            self.tree._lib.simlod_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
