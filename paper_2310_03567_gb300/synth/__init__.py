"""Seeded synthetic point clouds and batch cuts for the octree-update workloads.

The generator is plain C (``synth.c``) driven through ctypes. It holds no octree
arithmetic; its 16-byte records (int32 xyz in mm + RGBA8) are the input of both
the CUDA path and the CPU oracle. Every draw is addressed by position in a
SplitMix64 stream, so the output does not depend on the thread count.

Workloads (stand-ins for the paper's scans, Section 7.1):

* ``uniform``: points uniform in a cube (the 1 km, 1M-point case).
* ``aerial``: an fBm terrain sampled in scan-line order (aerial LIDAR-like).
* ``clustered``: points on random planar quads with log-normal density
  (terrestrial building scan-like), batches cut to random sizes and shuffled.
* ``mixed``: aerial and clustered runs interleaved, log-uniform batch sizes.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from .. import _build

POINT_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                        ("r", "u1"), ("g", "u1"), ("b", "u1"), ("a", "u1")])
assert POINT_DTYPE.itemsize == 16


class _TerrainParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("extent_m", ctypes.c_double),
                ("row_len", ctypes.c_uint32), ("wavelength_m", ctypes.c_double),
                ("octaves", ctypes.c_uint32), ("relief_m", ctypes.c_double),
                ("jitter_m", ctypes.c_double), ("offset_x_m", ctypes.c_double),
                ("offset_y_m", ctypes.c_double), ("coord_max", ctypes.c_int64)]


class _ClusterParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_quads", ctypes.c_uint32),
                ("n_points", ctypes.c_uint64), ("lo_m", ctypes.c_double * 3),
                ("hi_m", ctypes.c_double * 3), ("side_min_m", ctypes.c_double),
                ("side_max_m", ctypes.c_double), ("density_sigma", ctypes.c_double),
                ("noise_m", ctypes.c_double), ("coord_max", ctypes.c_int64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        u64, i64, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
        lib.synth_uniform.argtypes = [u64, i64, u64, u64, P, i32]
        lib.synth_terrain.argtypes = [ctypes.POINTER(_TerrainParams), u64, u64, P, i32]
        lib.synth_terrain_height01.argtypes = [ctypes.POINTER(_TerrainParams),
                                               ctypes.c_double, ctypes.c_double]
        lib.synth_terrain_height01.restype = ctypes.c_double
        lib.synth_cluster_counts.argtypes = [ctypes.POINTER(_ClusterParams), P]
        lib.synth_cluster_counts.restype = i32
        lib.synth_cluster_points.argtypes = [ctypes.POINTER(_ClusterParams), P, P, i32]
        lib.synth_batches.argtypes = [u64, u64, u64, u64, i32, P, P, u64]
        lib.synth_batches.restype = i64
        lib.synth_batches_loguniform.argtypes = [u64, u64, u64, u64, P, P, u64]
        lib.synth_batches_loguniform.restype = i64
        _lib = lib
    return _lib


def _threads(threads):
    return int(threads or os.cpu_count() or 1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def uniform(seed: int, extent: int, n: int, i0: int = 0, threads=None) -> np.ndarray:
    """Points i0..i0+n-1: x, y, z uniform integers in [0, extent), RGBA uniform."""
    out = np.empty(n, POINT_DTYPE)
    if n:
        _load().synth_uniform(seed, extent, i0, n, _ptr(out), _threads(threads))
    return out


def _terrain_params(seed, extent_m, row_len, root_log2, offset=(0.0, 0.0)):
    return _TerrainParams(seed, extent_m, row_len, 2000.0, 8, 300.0, 0.05,
                          offset[0], offset[1], (1 << root_log2) - 1)


def terrain(seed: int, n: int, i0: int = 0, extent_m: float = 4000.0, row_len: int = 7072,
            root_log2: int = 22, offset=(0.0, 0.0), threads=None) -> np.ndarray:
    """Points i0..i0+n-1 of the scan-line terrain stream."""
    out = np.empty(n, POINT_DTYPE)
    if n:
        P = _terrain_params(seed, extent_m, row_len, root_log2, offset)
        _load().synth_terrain(ctypes.byref(P), i0, n, _ptr(out), _threads(threads))
    return out


def _cluster_params(seed, n_quads, n_points, root_log2, lo=(15.0, 15.0, 15.0),
                    hi=(1985.0, 1985.0, 85.0)):
    P = _ClusterParams()
    P.seed, P.n_quads, P.n_points = seed, n_quads, n_points
    for k in range(3):
        P.lo_m[k], P.hi_m[k] = lo[k], hi[k]
    P.side_min_m, P.side_max_m = 0.5, 20.0
    P.density_sigma, P.noise_m = 1.5, 0.002
    P.coord_max = (1 << root_log2) - 1
    return P


def clustered(seed: int, n_quads: int, n_points: int, root_log2: int = 21,
              lo=(15.0, 15.0, 15.0), hi=(1985.0, 1985.0, 85.0), threads=None) -> np.ndarray:
    """All points of the quad set, quad by quad."""
    lib = _load()
    P = _cluster_params(seed, n_quads, n_points, root_log2, lo, hi)
    counts = np.empty(n_quads, np.uint64)
    if lib.synth_cluster_counts(ctypes.byref(P), _ptr(counts)) != 0:
        raise MemoryError("synth_cluster_counts failed")
    offsets = np.zeros(n_quads + 1, np.uint64)
    np.cumsum(counts, out=offsets[1:])
    out = np.empty(n_points, POINT_DTYPE)
    lib.synth_cluster_points(ctypes.byref(P), _ptr(offsets), _ptr(out), _threads(threads))
    return out


def batch_cut(seed: int, n: int, lo: int, hi: int, permute: bool):
    """Batch sizes uniform in [lo, hi]; returns (offsets, counts) in insertion order."""
    cap = n // max(lo, 1) + 2
    off = np.empty(cap, np.uint64)
    cnt = np.empty(cap, np.uint64)
    k = _load().synth_batches(seed, n, lo, hi, int(permute), _ptr(off), _ptr(cnt), cap)
    if k < 0:
        raise RuntimeError("batch table overflow")
    return off[:k].copy(), cnt[:k].copy()


def batch_cut_loguniform(seed: int, n: int, lo: int, hi: int):
    cap = n // max(lo, 1) + 2
    off = np.empty(cap, np.uint64)
    cnt = np.empty(cap, np.uint64)
    k = _load().synth_batches_loguniform(seed, n, lo, hi, _ptr(off), _ptr(cnt), cap)
    if k < 0:
        raise RuntimeError("batch table overflow")
    return off[:k].copy(), cnt[:k].copy()


@dataclasses.dataclass
class Workload:
    """A point stream with its root cube and its batch cut.

    ``points`` holds the records; batch k of the stream is
    ``points[offsets[k]:offsets[k]+counts[k]]`` and batches are inserted in
    list order, which fixes every point's global arrival index.
    """
    name: str
    points: np.ndarray
    offsets: np.ndarray
    counts: np.ndarray
    root_min: tuple
    root_log2: int
    recipe: str

    @property
    def n_points(self) -> int:
        return int(self.counts.sum())

    def batches(self):
        for o, c in zip(self.offsets, self.counts):
            yield self.points[int(o):int(o) + int(c)]

    def stream(self) -> np.ndarray:
        """The points in insertion order (a copy when batches are shuffled)."""
        if all(int(self.offsets[k]) == int(self.counts[:k].sum()) for k in range(len(self.counts))):
            return self.points[: self.n_points]
        return np.concatenate(list(self.batches()))


def _even_cut(n: int, batch: int):
    k = (n + batch - 1) // batch
    off = np.arange(k, dtype=np.uint64) * np.uint64(batch)
    cnt = np.minimum(np.uint64(batch), np.uint64(n) - off).astype(np.uint64)
    return off, cnt


def uniform_workload(n: int = 1_000_000, batch: int = 100_000, seed: int = 0,
                     extent: int = 1_000_000, root_log2: int = 20) -> Workload:
    pts = uniform(seed, extent, n)
    off, cnt = _even_cut(n, batch)
    return Workload(f"uniform-{n}", pts, off, cnt, (0, 0, 0), root_log2,
                    f"seed {seed}; {n} points, x/y/z uniform integer mm in [0,{extent}), "
                    f"RGBA uniform; batches of {batch}; root [0,2^{root_log2})^3")


def aerial_workload(n: int = 50_000_000, batch: int = 1_000_000, seed: int = 1) -> Workload:
    pts = terrain(seed, n)
    off, cnt = _even_cut(n, batch)
    return Workload(f"aerial-{n}", pts, off, cnt, (0, 0, 0), 22,
                    f"seed {seed}; 4 km x 4 km fBm terrain (8 octaves, 2 km base wavelength, "
                    f"300 m relief), scan lines of 7072 points, 5 cm jitter, first {n} points; "
                    f"batches of {batch}; root [0,2^22)^3 mm")


def clustered_workload(n: int = 300_000_000, n_quads: int = 20_000, seed: int = 2,
                       batch_lo: int = 1_000_000, batch_hi: int = 10_000_000) -> Workload:
    pts = clustered(seed, n_quads, n)
    off, cnt = batch_cut(seed, n, batch_lo, batch_hi, permute=True)
    return Workload(f"clustered-{n}", pts, off, cnt, (0, 0, 0), 21,
                    f"seed {seed}; {n_quads} planar quads, sides log-uniform 0.5-20 m, "
                    f"log-normal density (sigma 1.5), 2 mm noise, {n} points; batches "
                    f"uniform in [{batch_lo},{batch_hi}] in shuffled order; root [0,2^21)^3 mm")


def mixed_workload(n: int = 100_000_000, seed: int = 3, batch_lo: int = 65_536,
                   batch_hi: int = 8_388_608, run_lo: int = 1_000_000,
                   run_hi: int = 10_000_000) -> Workload:
    """Terrain and clustered points over one 4 km square, interleaved in runs."""
    half = n // 2
    ter = terrain(seed, half)
    clu = clustered(seed, max(1, (20_000 * half) // 300_000_000 or 1), n - half, root_log2=22,
                    lo=(15.0, 15.0, 15.0), hi=(3985.0, 3985.0, 285.0))
    r_off_t, r_cnt_t = batch_cut(seed + 101, half, run_lo, run_hi, permute=False)
    r_off_c, r_cnt_c = batch_cut(seed + 202, n - half, run_lo, run_hi, permute=False)
    parts = []
    for k in range(max(len(r_off_t), len(r_off_c))):
        if k < len(r_off_t):
            parts.append(ter[int(r_off_t[k]):int(r_off_t[k] + r_cnt_t[k])])
        if k < len(r_off_c):
            parts.append(clu[int(r_off_c[k]):int(r_off_c[k] + r_cnt_c[k])])
    pts = np.concatenate(parts)
    off, cnt = batch_cut_loguniform(seed, n, batch_lo, batch_hi)
    return Workload(f"mixed-{n}", pts, off, cnt, (0, 0, 0), 22,
                    f"seed {seed}; {half} terrain + {n - half} clustered points over a 4 km "
                    f"square, alternating runs of 1M-10M; batches log-uniform in "
                    f"[{batch_lo},{batch_hi}]; root [0,2^22)^3 mm")


def _spread3(v: np.ndarray) -> np.ndarray:
    """Bits 0..20 of v to bits 0, 3, 6, ..., 60 (Morton interleave)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_workload(w: Workload) -> Workload:
    """The same points and batch sizes, with the stream sorted in Morton
    (z-curve) order of the top 21 bits of each coordinate relative to the root
    (the paper's Morton-ordered input variant)."""
    pts = w.stream()
    shift = np.uint64(max(0, w.root_log2 - 21))
    key = np.zeros(len(pts), np.uint64)
    for a, f in enumerate("xyz"):
        rel = (pts[f].astype(np.int64) - int(w.root_min[a])).astype(np.uint64) >> shift
        key |= _spread3(rel) << np.uint64(a)
    order = np.argsort(key, kind="stable")
    sorted_pts = pts[order]
    cnt = w.counts.copy()
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64)
    return Workload(w.name + "-morton", sorted_pts, off, cnt, w.root_min, w.root_log2,
                    w.recipe + "; stream sorted in Morton order, same batch sizes in order")
