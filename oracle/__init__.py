"""CPU oracle for the incremental octree LOD update (SimLOD, Section 5).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only code allowed to import this package.
The product path (the CUDA library and its binding) never touches it.

Two plain C implementations (``incremental.c``, ``static.c``; see
``oracle.h`` for the readings of the paper they share) are driven through
ctypes and export the canonical octree as numpy structured arrays:

* ``nodes``: level, is_inner, min xyz, log2size, n_points, n_voxels, n_chunks,
  sorted by (level, ix, iy, iz);
* ``points``: x, y, z, rgba, gidx per leaf, sorted by gidx, leaves in node order;
* ``voxels``: cell, x, y, z, rgba per inner node, sorted by cell, in node order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_DIR, "liboracle.so")
_SOURCES = [os.path.join(_DIR, f) for f in ("incremental.c", "static.c", "render.c")]
_HEADER = os.path.join(_DIR, "oracle.h")

NODE_DTYPE = np.dtype([("level", "<u4"), ("is_inner", "<u4"), ("min", "<i4", (3,)),
                       ("log2size", "<u4"), ("n_points", "<u8"), ("n_voxels", "<u8"),
                       ("n_chunks", "<u8")])
POINT_REC_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("rgba", "<u4"),
                            ("gidx", "<u4")])
VOXEL_REC_DTYPE = np.dtype([("cell", "<u4"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                            ("rgba", "<u4")])
assert NODE_DTYPE.itemsize == 48 and POINT_REC_DTYPE.itemsize == 20
assert VOXEL_REC_DTYPE.itemsize == 20

OK, ERR_INVALID, ERR_OUT_OF_BOUNDS, ERR_NOMEM, ERR_ITER_CAP, ERR_TOO_MANY = 0, -1, -2, -3, -6, -11


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class Config(ctypes.Structure):
    """Octree parameters; defaults are the paper's (Sections 3.1, 3.3, 3.4)."""
    _fields_ = [("root_min", ctypes.c_int32 * 3), ("root_log2", ctypes.c_uint32),
                ("leaf_capacity", ctypes.c_uint32), ("chunk_points", ctypes.c_uint32),
                ("grid_log2", ctypes.c_uint32), ("max_expand_iters", ctypes.c_uint32)]

    @classmethod
    def make(cls, root_min=(0, 0, 0), root_log2=20, leaf_capacity=50_000, chunk_points=1_000,
             grid_log2=7, max_expand_iters=0):
        c = cls()
        for k in range(3):
            c.root_min[k] = int(root_min[k])
        c.root_log2, c.leaf_capacity, c.chunk_points = root_log2, leaf_capacity, chunk_points
        c.grid_log2, c.max_expand_iters = grid_log2, max_expand_iters
        return c


class _Sizes(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint64), ("n_points", ctypes.c_uint64),
                ("n_voxels", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "batches", "points", "spilled", "splits", "voxels", "iterations_max", "chunks_live",
        "chunks_pool", "chunks_bumped", "spill_voxels_at_old_inner")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved)."""
    stale = (not os.path.exists(_LIB_PATH) or
             any(os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SOURCES + [_HEADER]))
    if force or stale:
        tmp = _LIB_PATH + ".tmp"
        # no contraction: the renderer's float arithmetic is one IEEE operation
        # per written operator (so that the GPU can match it bit for bit)
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", *_SOURCES,
               "-o", tmp, "-lm"]
        proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if proc.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + proc.stdout)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        # a test may point this at a deliberately broken copy (mutation check)
        path = os.environ.get("SIMLOD_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P, u64 = ctypes.c_void_p, ctypes.c_uint64
        lib.orc_inc_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(P)]
        lib.orc_inc_insert.argtypes = [P, P, u64]
        lib.orc_inc_sizes.argtypes = [P, ctypes.POINTER(_Sizes)]
        lib.orc_inc_sizes.restype = None
        lib.orc_inc_export.argtypes = [P, P, P, P]
        lib.orc_inc_stats.argtypes = [P, ctypes.POINTER(Stats)]
        lib.orc_inc_stats.restype = None
        lib.orc_inc_destroy.argtypes = [P]
        lib.orc_inc_destroy.restype = None
        lib.orc_static_build.argtypes = [ctypes.POINTER(Config), P, u64, ctypes.POINTER(P)]
        lib.orc_static_sizes.argtypes = [P, ctypes.POINTER(_Sizes)]
        lib.orc_static_sizes.restype = None
        lib.orc_static_export.argtypes = [P, P, P, P]
        lib.orc_static_destroy.argtypes = [P]
        lib.orc_static_destroy.restype = None
        lib.orc_render.argtypes = [ctypes.POINTER(Config), P, u64, P, P, P, ctypes.c_uint32,
                                   ctypes.c_uint32, P, P, ctypes.POINTER(u64)]
        _lib = lib
    return _lib


class Snapshot:
    """Canonical octree: ``nodes``, ``points`` and ``voxels`` structured arrays."""

    def __init__(self, nodes, points, voxels):
        self.nodes, self.points, self.voxels = nodes, points, voxels

    def node_slices(self):
        """Yield (node record, its points, its voxels) in canonical order."""
        po = np.concatenate([[0], np.cumsum(self.nodes["n_points"])]).astype(np.int64)
        vo = np.concatenate([[0], np.cumsum(self.nodes["n_voxels"])]).astype(np.int64)
        for k in range(len(self.nodes)):
            yield (self.nodes[k], self.points[po[k]:po[k + 1]], self.voxels[vo[k]:vo[k + 1]])


def _as_points(pts) -> np.ndarray:
    a = np.ascontiguousarray(pts)
    if a.dtype.itemsize != 16:
        raise TypeError("points must be 16-byte records (int32 xyz + RGBA8)")
    return a


def _export(lib_export, handle, sizes: _Sizes) -> Snapshot:
    nodes = np.zeros(sizes.n_nodes, NODE_DTYPE)
    points = np.zeros(sizes.n_points, POINT_REC_DTYPE)
    voxels = np.zeros(sizes.n_voxels, VOXEL_REC_DTYPE)
    rc = lib_export(handle, nodes.ctypes.data, points.ctypes.data, voxels.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "export")
    return Snapshot(nodes, points, voxels)


class Incremental:
    """The per-batch update of Section 5, sequential on one core."""

    def __init__(self, config: Config):
        self._lib = _load()
        self._h = ctypes.c_void_p()
        rc = self._lib.orc_inc_create(ctypes.byref(config), ctypes.byref(self._h))
        if rc != OK:
            raise OracleError(rc, "create")
        self.config = config

    def insert(self, pts) -> int:
        """Insert one batch; returns the oracle status (0 = applied)."""
        a = _as_points(pts)
        return self._lib.orc_inc_insert(self._h, a.ctypes.data if len(a) else None, len(a))

    def snapshot(self) -> Snapshot:
        s = _Sizes()
        self._lib.orc_inc_sizes(self._h, ctypes.byref(s))
        return _export(self._lib.orc_inc_export, self._h, s)

    def stats(self) -> dict:
        st = Stats()
        self._lib.orc_inc_stats(self._h, ctypes.byref(st))
        return st.as_dict()

    def close(self):
        if self._h:
            self._lib.orc_inc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def static_build(config: Config, pts) -> Snapshot:
    """The closed-form octree of a whole prefix (static.c)."""
    lib = _load()
    a = _as_points(pts)
    h = ctypes.c_void_p()
    rc = lib.orc_static_build(ctypes.byref(config), a.ctypes.data if len(a) else None, len(a),
                              ctypes.byref(h))
    if rc != OK:
        raise OracleError(rc, "static build")
    try:
        s = _Sizes()
        lib.orc_static_sizes(h, ctypes.byref(s))
        return _export(lib.orc_static_export, h, s)
    finally:
        lib.orc_static_destroy(h)


def incremental_build(config: Config, batches) -> tuple[Snapshot, dict]:
    """Insert every batch in order; returns the final snapshot and the stats."""
    o = Incremental(config)
    try:
        for b in batches:
            rc = o.insert(b)
            if rc != OK:
                raise OracleError(rc, "insert")
        return o.snapshot(), o.stats()
    finally:
        o.close()


def render(cfg: Config, snap: Snapshot, view_proj, width: int, height: int):
    """Section 6 on the CPU: returns (framebuffer as uint64 [height, width],
    per-node drawn flags in canonical order, number of drawn nodes).
    view_proj: 16 float32, row-major; see render.c for the readings."""
    lib = _load()
    m = np.ascontiguousarray(np.asarray(view_proj, dtype=np.float32).reshape(16))
    nodes = np.ascontiguousarray(snap.nodes)
    points = np.ascontiguousarray(snap.points)
    voxels = np.ascontiguousarray(snap.voxels)
    fb = np.empty((height, width), np.uint64)
    drawn = np.zeros(len(nodes), np.uint8)
    nd = ctypes.c_uint64()
    rc = lib.orc_render(ctypes.byref(cfg), nodes.ctypes.data, len(nodes), points.ctypes.data,
                        voxels.ctypes.data, m.ctypes.data, width, height, fb.ctypes.data,
                        drawn.ctypes.data, ctypes.byref(nd))
    if rc != OK:
        raise OracleError(rc, "orc_render")
    return fb, drawn.astype(bool), int(nd.value)
