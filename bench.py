#!/usr/bin/env python3
"""Throughput of the incremental octree LOD update on one GB300 per rank.

One step = one pass of the whole update path over the workload: reset the
octree, then insert every batch of the stream (count, split, voxel claim,
chunk allocation, scatter) with the batches already resident in HBM. The
default workload is the 300M-point clustered building scan, cut into batches
of 1M-10M points in shuffled order, applied by one persistent launch per step.

The default run (one GPU) adds the two forms built on the update to the same
line: `batched` (the 100M-point mixed stream in uneven batches of 64k-8M
points: the autotuned plan against the same batches one launch per step and
through the plain per-kernel path) and `serving` (16 resident octrees served
from Poisson request traces against a plain server, latency p50/p99 and
throughput).

Prints one JSON line (rank 0). With --impl reference the CPU oracle is timed
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

REPO = os.path.dirname(os.path.abspath(__file__))
if REPO not in sys.path:
    sys.path.insert(0, REPO)

METRIC = "Mpts/s inserted into octree (frac. of HBM roofline); p50/p99 batch latency vs plain"
UNIT = "Mpts/s"
L2_BYTES = 129 << 20
CTL_BYTES = 256  # the library's control block, read once per expansion round

# Algorithmic bytes of one update: read every batch point (16 B), write
# every point with its gidx (20 B), read and rewrite every re-inserted point
# (2 x 20 B), write every new voxel (16 B), zero one grid per split. Repeated
# traversals, cursors, the claim table and the backlog are implementation
# overhead and are not counted.


def update_alg_bytes(B, S, V, K, grid_bytes):
    return 16 * B + 20 * B + 40 * S + 16 * V + grid_bytes * K


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_fused
# launch over a whole workload (every batch of the stream: the launch the
# bench times), from an ncu capture of that launch with the DRAM byte
# counters alone (one pass, so nothing is replayed). Keyed by a hash of the
# kernel's sources and by the workload: a changed kernel reports null until
# it has been captured again.
KERNEL_SOURCES = ("paper_2310_03567_gb300/csrc/device.cuh", "paper_2310_03567_gb300/csrc/fused.cuh",
                  "include/simlod.h", "paper_2310_03567_gb300/_build.py")
TRAFFIC_PER_LAUNCH = {
    # clustered-300M, one launch over its 54 batches: 39.07 GB read + 23.29 GB
    # written in 49.63 ms (profiles/k_fused_clustered300m_dram.md)
    ("b05ed5b4e3dd2b94", "clustered-300000000"): 62.36e9,
}


def paper_style_roofline(B, S, V, K, grid_bytes, peak_gbs, mpts):
    """The same roofline with the paper's 16-byte records only (no 4-byte
    gidx stored beside each point): 16 B read + 16 B written per point, 32 B
    per re-inserted point."""
    b = 16 * B + 16 * B + 32 * S + 16 * V + grid_bytes * K
    roof = B / (b / (peak_gbs * 1e9)) / 1e6
    return {"alg_bytes_per_point": b / B, "roofline_mpts": roof, "frac": mpts / roof}


def host_cpu() -> dict:
    """The host's CPU model and core count (for the CPU oracle's numbers)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model name"):
                    model = v.strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                k, _, v = line.partition(":")
                if k.strip() == "Model name":
                    model = v.strip()
                    break
        except Exception:
            pass
    return {"model": model or platform.processor() or "unknown", "arch": platform.machine(),
            "nproc": os.cpu_count()}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(REPO, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_workload(name: str, points: int | None, morton: bool = False):
    from paper_2310_03567_gb300 import synth
    if morton:
        w, root = make_workload(name, points)
        return synth.morton_workload(w), root
    if name == "aerial":
        return synth.aerial_workload(n=points or 50_000_000), 22
    if name == "uniform":
        return synth.uniform_workload(n=points or 1_000_000), 20
    if name == "clustered":
        return synth.clustered_workload(n=points or 300_000_000), 21
    if name == "mixed":
        return synth.mixed_workload(n=points or 100_000_000), 22
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(workload, budget_s: float = 12.0):
    """The incremental oracle on the host, one core, on the first batches of the
    workload until the time budget is used (at least one batch)."""
    import oracle
    w, root_log2 = workload
    cfg = oracle.Config.make(root_min=w.root_min, root_log2=root_log2)
    inc = oracle.Incremental(cfg)
    pts = 0
    t0 = time.perf_counter()
    nb = 0
    for b in w.batches():
        rc = inc.insert(b)
        if rc != oracle.OK:
            raise RuntimeError(f"oracle insert failed: {rc}")
        pts += len(b)
        nb += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    inc.close()
    return {"value": pts / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {nb} batches ({pts} points) of {w.name}, sequential incremental "
                      f"oracle, {dt:.1f} s", "host": host_cpu()}


def workload_config(w, max_batch: int, world: int) -> dict:
    """The `config` object of the JSON line: the workload, its cut and the
    octree parameters (the same for both arms)."""
    return {"workload": w.name, "batch_points": int(max_batch),
            "batches_per_step": len(w.counts), "points_per_step": w.n_points,
            "leaf_capacity": 50_000, "chunk_points": 1000, "grid": 128,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (%.0f MB of points)" % (w.n_points * 16 / 2**20)}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on the host cores, on a
    bounded sample of the same workload (its first batches, at least
    --ref-points points) per step."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    # the serving trace's octrees are terrain / uniform / clustered streams;
    # the oracle is timed on the terrain (aerial) stream for it
    workload = make_workload("aerial" if args.workload == "serving" else args.workload,
                             args.points)
    w, root_log2 = workload
    import oracle
    cfg = oracle.Config.make(root_min=w.root_min, root_log2=root_log2)
    nb, pts = 0, 0
    while nb < len(w.counts) and (nb == 0 or pts < args.ref_points):
        pts += int(w.counts[nb])
        nb += 1
    sample = list(w.batches())[:nb]

    def step():
        inc = oracle.Incremental(cfg)
        for b in sample:
            assert inc.insert(b) == oracle.OK
        inc.close()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = pts * args.steps / dt / 1e6
    what = (f"first {nb} batches ({pts} points) of {w.name} per step, sequential incremental "
            f"oracle on one host core")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(w, max(int(c) for c in w.counts), world),
            "sample": {"batches_per_step": nb, "points_per_step": pts},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": what, "host": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def make_octree(w, root_log2: int, chunk_points: int = 1000, max_batch: int | None = None):
    """The octree the bench times for workload w (its capacities follow the
    workload's largest batch, or max_batch: the batched form merges batches
    into updates of up to that size); the full-size tests build the same one."""
    import torch

    from paper_2310_03567_gb300 import simlod
    max_batch = max(int(max(w.counts)), int(max_batch or 0))
    # claim table: 2 slots per backlog entry. Up to 2 new voxels per batch
    # point, but at most 8M per update (these workloads make under 5M new
    # voxels in any one update): the table (64-256 MB) stays mostly
    # L2-resident instead of a 1 GB table for 10M-point batches
    cfg = simlod.default_config(root_min=w.root_min, root_log2=root_log2,
                                max_batch_points=max_batch,
                                spill_capacity=max(8 << 20, 2 * max_batch),
                                backlog_capacity=max(2 << 20, min(2 * max_batch, 8 << 20)),
                                max_nodes=1 << 21, chunk_points=chunk_points)
    # plus the part-filled last chunk of up to 64k nodes
    data_bytes = max(256 << 20, w.n_points * 80) + (1 << 16) * 20 * chunk_points
    arena = simlod.make_arena(cfg, data_bytes)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    return simlod.Octree(cfg, arena, stream=stream)


def rank_workload(name: str, points, rank: int, morton: bool = False):
    """The workload a rank builds: every rank has its own octree and stream
    (independent units, no data-path collective); rank r > 0 gets its own
    seed so that the replicas are not copies."""
    w, root_log2 = make_workload(name, points, morton)
    if rank:
        from paper_2310_03567_gb300 import synth
        if name == "aerial":
            w.points = synth.terrain(1 + 1000 * rank, w.n_points)
        elif name == "uniform":
            w.points = synth.uniform(1000 * rank, 1_000_000, w.n_points)
        elif name == "clustered":
            w = synth.clustered_workload(n=w.n_points, seed=2 + 1000 * rank)
    return w, root_log2


def prefix_workload(w, k: int):
    """The first k batches of workload w, as a workload of their own (the
    points of those batches only, in insertion order)."""
    from paper_2310_03567_gb300 import synth
    k = max(1, min(k, len(w.counts)))
    pts = np.concatenate([w.points[int(o):int(o) + int(c)]
                          for o, c in zip(w.offsets[:k], w.counts[:k])])
    cnt = w.counts[:k].copy()
    off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64)
    return synth.Workload(f"{w.name}-first{k}", pts, off, cnt, w.root_min, w.root_log2,
                          w.recipe + f"; its first {k} batches")


def aggregate(ms_local: float, points_local: int, dist=None, device="cpu"):
    """Whole-job timing across ranks: the slowest rank's time and the total
    points of all ranks (value = total / max time)."""
    if dist is None:
        return ms_local, points_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    p = torch.tensor([points_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), int(p.item())


def percentile(v, q):
    if not v:
        return None
    s = sorted(v)
    k = min(len(s) - 1, max(0, int(round(q / 100.0 * (len(s) - 1)))))
    return s[k]


def run_ours(args):
    import torch

    from paper_2310_03567_gb300 import simlod

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    simlod.load()

    # each rank builds its own octree from its own stream (independent units)
    w, root_log2 = rank_workload(args.workload, args.points, rank, args.morton)
    if args.batches:  # a prefix of the stream (profiling of a small case)
        w = prefix_workload(w, args.batches)
    n_points = w.n_points
    dev_pts = simlod.points_tensor(w.points)
    ptrs = [dev_pts.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    max_batch = max(counts)
    tree = make_octree(w, root_log2, max_batch=args.max_batch)
    cfg = tree.cfg
    stream = tree.stream

    def check(rc, what):
        if rc != simlod.OK:
            raise simlod.SimlodError(rc, what)

    def fused_step():
        tree.reset()
        check(tree.insert_many_ptrs(ptrs, counts), "insert_batches")

    def plain_pass(lat=None):
        tree.reset()
        for ptr, cnt in zip(ptrs, counts):
            if lat is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            check(tree.insert_ptr(ptr, cnt), "insert_batch")
            if lat is not None:
                b.record(stream)
                lat.append((a, b))

    for _ in range(args.warmup):
        fused_step()
    check(tree.sync(), "warm-up")
    stats = tree.stats()  # counts of one full pass

    # ---- timed region: K steps of the fused form
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    tree.set_timing(True, clear=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        fused_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    tree.set_timing(False)
    clk = clocks.stop()
    check(tree.sync(), "timed steps")
    ms_total, job_points = aggregate(ev0.elapsed_time(ev1), n_points, dist, "cuda")
    if dist:
        dist.barrier()
    ktime = tree.timing()
    phases = {k: v / args.steps for k, v in tree.phase_times().items() if v > 0}

    # ---- per-batch latency: fused form one launch per batch, and plain form
    lat_fused = []
    tree.reset()
    for ptr, cnt in zip(ptrs, counts):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        check(tree.insert_many_ptrs([ptr], [cnt]), "insert_batches")
        b.record(stream)
        lat_fused.append((a, b))
    check(tree.sync(), "latency (fused)")
    lat_plain = []
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    plain_pass()  # warm
    check(tree.sync(), "plain warm-up")
    tree.set_timing(True, clear=True)
    pe0.record(stream)
    plain_pass(lat_plain)
    pe1.record(stream)
    torch.cuda.synchronize()
    tree.set_timing(False)
    check(tree.sync(), "plain pass")
    plain_ms = pe0.elapsed_time(pe1)
    plain_k = {k: v[1] for k, v in tree.timing().items() if v[0]}
    lat_f = [a.elapsed_time(b) for a, b in lat_fused]
    lat_p = [a.elapsed_time(b) for a, b in lat_plain]

    # ---- one 1920x1080 frame of the whole octree (Section 6 renderer), from
    # an oblique overview camera
    side = float(1 << root_log2)
    ctr = np.asarray(w.root_min, float) + side * np.array([0.5, 0.5, 0.02])
    eye = ctr + side * np.array([-0.45, -0.55, 0.35])
    cam = simlod.view_proj(eye, ctr, 60.0, 1920 / 1080)
    frame = torch.empty((1080, 1920), dtype=torch.int64, device="cuda")
    for _ in range(2):
        tree.render(cam, frame)
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(5):
        tree.render(cam, frame)
    r1.record(stream)
    torch.cuda.synchronize()
    check(tree.sync(), "render")
    rst = tree.stats()
    render = {"ms": r0.elapsed_time(r1) / 5, "width": 1920, "height": 1080,
              "nodes": rst["render_nodes"], "samples": rst["render_samples"],
              "pixels_hit": int((frame != -1).sum().item())}
    # ---- compaction of every node into a contiguous array (simlod_compact),
    # and the same frame again
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    before = frame.clone()
    c0.record(stream)
    tree.compact(0)
    c1.record(stream)
    tree.render(cam, frame)
    r0.record(stream)
    for _ in range(5):
        tree.render(cam, frame)
    r1.record(stream)
    torch.cuda.synchronize()
    check(tree.sync(), "compact")
    cst = tree.stats()
    render["compacted"] = {"compact_ms": c0.elapsed_time(c1), "nodes": cst["compact_nodes"],
                           "chunks_freed": cst["compact_chunks_freed"],
                           "render_ms": r0.elapsed_time(r1) / 5,
                           "same_frame": bool(torch.equal(before, frame))}
    del frame, before

    # ---- end to end through the public API: pinned host stream -> HBM,
    # fused update, result (stats) back to the host, every step
    host_pts = torch.from_numpy(np.ascontiguousarray(w.points).view(np.uint8).reshape(-1, 16))
    host_pts = host_pts.pin_memory()
    dev_e2e = torch.empty_like(dev_pts)
    e2e_ptrs = [dev_e2e.data_ptr() + int(o) * 16 for o in w.offsets]

    def e2e_step():
        with torch.cuda.stream(stream):
            dev_e2e.copy_(host_pts, non_blocking=True)
        tree.reset()
        check(tree.insert_many_ptrs(e2e_ptrs, counts), "insert_batches (e2e)")
        return tree.stats()

    # pipelined: the batch list in groups of about 1/8, each group copied on
    # a copy stream while the update of the group before runs
    copy_stream = torch.cuda.Stream()
    groups = np.array_split(np.arange(len(ptrs)), min(8, len(ptrs)))

    def e2e_pipelined_step():
        tree.reset()
        for g in groups:
            lo, hi = int(w.offsets[g[0]]), int(w.offsets[g[-1]] + w.counts[g[-1]])
            with torch.cuda.stream(copy_stream):
                dev_e2e[lo:hi].copy_(host_pts[lo:hi], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
            stream.wait_event(ev)
            check(tree.insert_many_ptrs([e2e_ptrs[k] for k in g], [counts[k] for k in g]),
                  "insert_batches (e2e pipelined)")
        copy_stream.wait_stream(stream)  # the next step's copies overwrite this one's input
        return tree.stats()

    # direct: the persistent kernel reads the batches from pinned host memory
    # over the CPU-GPU link (no staging copy)
    host_ptrs = [host_pts.data_ptr() + int(o) * 16 for o in w.offsets]

    def e2e_direct_step():
        tree.reset()
        check(tree.insert_many_ptrs(host_ptrs, counts), "insert_batches (e2e direct)")
        return tree.stats()

    # host-fed: one persistent launch; each batch is copied on the copy stream
    # and the launch starts it once its ready flag is set (per-batch overlap)
    host_parts = [host_pts[int(o):int(o) + int(c)] for o, c in zip(w.offsets, w.counts)]
    ready = torch.empty(len(host_parts), dtype=torch.int32, device="cuda")

    def e2e_host_fed_step():
        tree.reset()
        tree.insert_many_host(host_parts, dev_e2e, ready, copy_stream)
        copy_stream.wait_stream(stream)  # the next step's copies overwrite this one's input
        return tree.stats()

    # every step is timed on its own (each ends with the stats read, so the
    # device is idle between steps); a mode's time is its median step
    e2e_steps = max(3, min(args.steps, 5))
    e2e_times, e2e_step_ms = {}, {}
    for name, fn in (("copy_then_update", e2e_step), ("pipelined", e2e_pipelined_step),
                     ("direct", e2e_direct_step), ("host_fed", e2e_host_fed_step)):
        fn()
        torch.cuda.synchronize()
        steps_s = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            st_e2e = fn()
            steps_s.append(time.perf_counter() - t0)
            if st_e2e["points"] != n_points:
                raise RuntimeError(f"e2e {name}: {st_e2e['points']} points applied")
        e2e_times[name] = statistics.median(steps_s)
        e2e_step_ms[name] = [round(x * 1e3, 2) for x in steps_s]
    e2e_mode = min(e2e_times, key=e2e_times.get)
    e2e_s = e2e_times[e2e_mode]
    del host_pts, dev_e2e, host_parts, ready

    # ---- roofline of the dominant kernel (the fused update: one launch = one step)
    peak, peak_src = load_peaks()
    B, S, V, K = n_points, stats["spilled"], stats["voxels"], stats["splits"]
    grid_bytes = (1 << (3 * cfg.grid_log2)) // 8
    upd_bytes = update_alg_bytes(B, S, V, K, grid_bytes)
    f_launches, f_ms = ktime["fused_update"]
    avg_ms = f_ms / max(f_launches, 1)
    achieved = upd_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms else 0.0
    ms_per_step = ms_total / args.steps
    value = job_points * args.steps / (ms_total * 1e-3) / 1e6
    path = "fused persistent launch per step (every batch a full update)"

    # ---- batched form (uneven batches): autotuned plan (merged updates, one
    # persistent launch, replayed as a CUDA graph), timed like the fused form
    batched = None
    if args.workload == "mixed" or args.batched:
        best, tune_ms = tree.autotune(ptrs, counts)
        plan = tree.plan(ptrs, counts, merge_points=best.merge_points,
                         blocks_per_sm=best.blocks_per_sm, use_graph=True,
                         variant=best.variant)
        params, graphed = plan.info()
        for _ in range(args.warmup):
            tree.reset()
            check(plan.run(), "plan run")
        check(tree.sync(), "batched warm-up")
        bstats = tree.stats()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            tree.reset()
            check(plan.run(), "plan run")
        b1.record(stream)
        torch.cuda.synchronize()
        check(tree.sync(), "batched steps")
        plan.close()
        b_ms, b_points = aggregate(b0.elapsed_time(b1), n_points, dist, "cuda")
        batched = {"value": b_points * args.steps / (b_ms * 1e-3) / 1e6, "unit": UNIT,
                   "ms_per_step": b_ms / args.steps, "params": params, "graph": graphed,
                   "updates_per_step": bstats["batches"], "autotune_best_ms": tune_ms,
                   "vs_fused_unmerged": None, "vs_plain": None}
        batched["vs_fused_unmerged"] = batched["value"] / value
        path = ("batched form: autotuned plan (merged updates, one persistent launch, "
                "CUDA graph) per step")
        fused_unmerged = {"value": value, "ms_per_step": ms_per_step}
        value, ms_per_step = batched["value"], batched["ms_per_step"]
    roofline_mpts = B / (upd_bytes / (peak * 1e9)) / 1e6
    traffic = TRAFFIC_PER_LAUNCH.get((kernel_source_hash(), w.name))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": workload_config(w, max_batch, world),
        "path": path,
        "latency_ms": {"fused_p50": percentile(lat_f, 50), "fused_p99": percentile(lat_f, 99),
                       "plain_p50": percentile(lat_p, 50), "plain_p99": percentile(lat_p, 99),
                       "batches": len(lat_f)},
        "plain": {"value": n_points / (plain_ms * 1e-3) / 1e6, "unit": UNIT,
                  "ms_per_step": plain_ms, "kernels_ms_per_step": plain_k},
        "roofline": {"bound": "hbm", "kernel": "k_fused", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "alg_bytes_per_launch": upd_bytes, "peak_source": peak_src},
        "update_roofline": {"alg_bytes_per_point": upd_bytes / B, "roofline_mpts": roofline_mpts,
                            "frac": value / world / roofline_mpts,
                            "paper_style": paper_style_roofline(B, S, V, K, grid_bytes,
                                                                peak, value / world)},
        "update_counts": {"B": B, "S": S, "V": V, "K": K, "rounds": stats["rounds"],
                          "nodes": stats["nodes"]},
        "fused_phase_ms_per_step": phases,
        "render_1080p": render,
        "batched": batched,
        "gpu_launches": 2 * args.steps,
        "e2e": {"value": job_points / e2e_s / 1e6, "unit": UNIT,
                # points, the batch table (24 B per batch) and, host-fed, a
                # 4-byte ready flag per batch
                "h2d_bytes_per_step": n_points * 16 + 24 * len(ptrs)
                + (4 * len(ptrs) if e2e_mode == "host_fed" else 0),
                "d2h_bytes_per_step": CTL_BYTES, "mode": e2e_mode,
                "timing": f"median of {e2e_steps} steps, each from the host's clock",
                "modes_mpts": {k: n_points / v / 1e6 for k, v in e2e_times.items()},
                "modes_step_ms": e2e_step_ms},
        "clocks": clk,
    }
    if batched is not None:
        batched["vs_plain"] = batched["value"] / line["plain"]["value"]
        line["fused_unmerged"] = fused_unmerged
        # merged updates re-insert fewer stored points: their own bytes per point
        b_alg = update_alg_bytes(B, bstats["spilled"], V, K, grid_bytes)
        b_roof = B / (b_alg / (peak * 1e9)) / 1e6
        line["update_roofline"] = {"alg_bytes_per_point": b_alg / B, "roofline_mpts": b_roof,
                                   "frac": value / world / b_roof, "form": "batched"}
        line["update_counts"]["S_batched"] = bstats["spilled"]
    tree.close()
    del tree, dev_pts
    torch.cuda.empty_cache()
    forms = args.forms and args.workload == "clustered" and not args.morton and not args.batches
    if forms and world == 1:
        # the two forms built on the update, each on its own workload
        line["batched"] = batched_form(args)
        torch.cuda.empty_cache()
        line["serving"] = serving_form(args)
        torch.cuda.empty_cache()
    elif forms:
        line["forms"] = "the batched and serving forms are measured in the one-GPU run"
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline((w, root_log2), args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batched_form(args) -> dict:
    """The batched form on the 100M-point mixed stream (terrain and clustered
    runs, batches log-uniform in 64k-8M points): the autotuned plan (merged
    updates, one persistent launch, CUDA-graph replay) against the same
    batches applied one update each in one persistent launch, and through the
    plain per-kernel path; per-batch latency of the fused form (one launch per
    batch) against the plain form."""
    import torch

    from paper_2310_03567_gb300 import simlod
    w, root_log2 = make_workload("mixed", None)
    dev = simlod.points_tensor(w.points)
    ptrs = [dev.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    tree = make_octree(w, root_log2)
    stream = tree.stream

    def check(rc, what):
        if rc != simlod.OK:
            raise simlod.SimlodError(rc, what)

    def timed(step, k):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    best, tune_ms = tree.autotune(ptrs, counts)
    plan = tree.plan(ptrs, counts, merge_points=best.merge_points,
                     blocks_per_sm=best.blocks_per_sm, use_graph=True,
                     variant=best.variant)
    params, graphed = plan.info()

    def plan_step():
        tree.reset()
        check(plan.run(), "plan run")

    def fused_step():
        tree.reset()
        check(tree.insert_many_ptrs(ptrs, counts), "insert_batches")

    lat_p = []

    def plain_step(lat=None):
        tree.reset()
        for ptr, cnt in zip(ptrs, counts):
            if lat is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            check(tree.insert_ptr(ptr, cnt), "insert_batch")
            if lat is not None:
                b.record(stream)
                lat.append((a, b))

    for _ in range(args.warmup):
        plan_step()
    check(tree.sync(), "batched warm-up")
    updates = tree.stats()["batches"]
    spilled = tree.stats()["spilled"]
    plan_ms = timed(plan_step, args.steps)
    check(tree.sync(), "batched steps")
    plan.close()
    for _ in range(args.warmup):
        fused_step()
    fused_ms = timed(fused_step, args.steps)
    check(tree.sync(), "fused steps")
    plain_step()
    plain_ms = timed(lambda: plain_step(lat_p), 1)
    check(tree.sync(), "plain pass")
    # per-batch latency of the fused form: each batch its own launch
    tree.reset()
    lat_f = []
    for ptr, cnt in zip(ptrs, counts):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        check(tree.insert_many_ptrs([ptr], [cnt]), "insert_batches")
        b.record(stream)
        lat_f.append((a, b))
    check(tree.sync(), "latency (fused)")
    torch.cuda.synchronize()
    lf = [a.elapsed_time(b) for a, b in lat_f]
    lp = [a.elapsed_time(b) for a, b in lat_p]
    tree.close()
    n = w.n_points
    out = {"workload": w.name, "batches": len(counts), "batch_points": "log-uniform 64k-8M",
           "value": n / (plan_ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": plan_ms,
           "params": params, "graph": graphed, "updates_per_step": updates,
           "spilled_per_step": spilled, "autotune_best_ms": tune_ms,
           "fused_unmerged": {"value": n / (fused_ms * 1e-3) / 1e6, "ms_per_step": fused_ms},
           "plain": {"value": n / (plain_ms * 1e-3) / 1e6, "ms_per_step": plain_ms},
           "latency_ms": {"fused_p50": percentile(lf, 50), "fused_p99": percentile(lf, 99),
                          "plain_p50": percentile(lp, 50), "plain_p99": percentile(lp, 99)}}
    out["vs_fused_unmerged"] = out["value"] / out["fused_unmerged"]["value"]
    out["vs_plain"] = out["value"] / out["plain"]["value"]
    return out


def serving_setup(scale: float, seed: int = 4):
    """The serving configuration: 16 octrees (sizes log-uniform in
    [5M, 200M] points times `scale`; uniform / terrain / clustered in turn),
    each with its own stream, arena and overview camera."""
    import torch

    from paper_2310_03567_gb300 import serving, simlod, synth
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(5e6), np.log(2e8), 16)) * scale
    streams, specs = [], []
    for k, n in enumerate(int(max(1000, s)) for s in sizes):
        kind = ("uniform", "terrain", "clustered")[k % 3]
        if kind == "uniform":
            pts, root = synth.uniform(seed * 100 + k, 1 << 20, n), 20
        elif kind == "terrain":
            pts, root = synth.terrain(seed * 100 + k, n), 22
        else:
            quads = max(50, int(20_000 * n / 300e6))
            pts, root = synth.clustered(seed * 100 + k, quads, n), 21
        side = float(1 << root)
        ctr = side * np.array([0.5, 0.5, 0.05])
        cam = simlod.view_proj(ctr + side * np.array([-0.45, -0.55, 0.35]), ctr, 60.0, 16 / 9)
        # a uniform octree can split a whole level at once: every stored
        # point may be re-inserted in one update, and each may make a voxel
        cap = min(max(16 << 20, n + 5_000_000), (1 << 31) - 1)
        cfg = simlod.default_config(root_log2=root, max_batch_points=5_000_000,
                                    spill_capacity=cap, backlog_capacity=cap, max_nodes=1 << 20)
        specs.append(serving.OctreeSpec(cfg, max(256 << 20, n * 80), cam))
        host = torch.from_numpy(pts.view(np.uint8).reshape(-1, 16)).pin_memory()
        streams.append(host)
    return streams, specs


def serving_form(args, rank: int = 0) -> dict:
    """Serving form: a saturated run of each server first queues a whole
    trace at once; then requests (log-uniform 100k-5M points) arrive by a
    Poisson process at 70 % of the plain server's saturated throughput on
    that trace; the same traces are served by the serving form and by a plain
    server (one request per update, one update at a time), taking turns trace
    by trace; each server serves its trace once untimed, then timed. Latency
    percentiles pool the requests of the timed traces."""
    import torch

    from paper_2310_03567_gb300 import serving, simlod
    streams, specs = serving_setup(args.serving_scale, seed=4 + rank)
    total = sum(int(s.shape[0]) for s in streams)
    arenas = sum(simlod.arena_bytes(sp.cfg, sp.data_bytes) for sp in specs)
    budget = arenas + (4 << 30)
    # saturated: a whole trace queued at once (throughput at capacity); the
    # plain server's saturated throughput on this very trace is the capacity
    # that sets the arrival rate of the timed traces (each server is built,
    # serves the trace once untimed, then once timed)
    cut = serving.poisson_requests(streams, 100_000, 5_000_000, 1e9, seed=7)
    sat = {}
    for name, plain in (("plain", True), ("serving", False)):
        srv = serving.Server(specs, hbm_budget=budget, compute_slots=2, frame_ms=33.3,
                             plain=plain)
        for warm in (True, False):
            for r in cut:
                r.admitted = r.launched = r.done = -1.0
                r.arrival = 0.0
            srv.reset()
            srv.run(cut)
        rep = srv.report()
        sat[name] = {"mpts_per_s": rep["mpts_per_s"], "seconds": rep["seconds"],
                     "launches": rep["launches"], "frames": rep["frames"]}
        srv.close()
        del srv
        torch.cuda.empty_cache()
    sat["serving_vs_plain"] = sat["serving"]["mpts_per_s"] / sat["plain"]["mpts_per_s"]
    cap = sat["plain"]["mpts_per_s"] * 1e6
    rate = 0.7 * cap
    # several independent Poisson traces (each the whole stream of every
    # octree); latency percentiles pool their requests, since a p99 over one
    # trace rests on its two or three slowest requests
    traces = [serving.poisson_requests(streams, 100_000, 5_000_000, rate, seed=7 + t)
              for t in range(args.serving_traces)]
    reqs = traces[0]
    out = {}
    clk = None
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    # the two servers take turns, one trace each, the first of each turn
    # alternating, so that a box that drifts during the run (some get slower
    # over minutes) weighs on both alike; every server is built for its trace
    # and serves it once untimed first (the first run after a build is slower)
    meas = {"serving": ([], [], [], [], [], [], [], []),
            "plain": ([], [], [], [], [], [], [], [])}
    for t, tr in enumerate(traces):
        order = (("serving", False), ("plain", True))
        for name, plain in (order if t % 2 == 0 else order[::-1]):
            lat, wait, reps, lwait, serv, slow, slow_l, slow_r = meas[name]
            srv = serving.Server(specs, hbm_budget=budget, compute_slots=2, frame_ms=33.3,
                                 plain=plain)
            for warm in (True, False):
                for r in tr:
                    r.admitted = r.launched = r.done = -1.0
                srv.reset()
                if not warm and not plain and t == 0:
                    clocks.start()
                done = srv.run(tr)
                if not warm and not plain and t == 0:
                    clk = clocks.stop()
            lat += [(r.done - r.arrival) * 1e3 for r in done]
            wait += [(r.admitted - r.arrival) * 1e3 for r in done]
            lwait += [(r.launched - r.admitted) * 1e3 for r in done]
            serv += [(r.done - r.launched) * 1e3 for r in done]
            reps.append(srv.report())
            slow += [dict(x, trace=t) for x in reps[-1]["slowest"]]
            slow_l += [dict(x, trace=t) for x in reps[-1]["slowest_launches"]]
            slow_r += [dict(x, trace=t) for x in reps[-1]["slowest_renders"]]
            srv.close()
            del srv
            torch.cuda.empty_cache()
    for name in ("serving", "plain"):
        lat, wait, reps, lwait, serv, slow, slow_l, slow_r = meas[name]
        rep = dict(reps[0])
        # frames and scheduler figures are the first trace's; latencies,
        # waits and service times pool every timed trace's requests
        rep["launch_wait_ms"] = {"p50": float(np.percentile(lwait, 50)),
                                 "p99": float(np.percentile(lwait, 99))}
        rep["service_ms"] = {"p50": float(np.percentile(serv, 50)),
                             "p99": float(np.percentile(serv, 99))}
        rep["slowest"] = sorted(slow, key=lambda x: -x["latency_ms"])[:8]
        rep["slowest_launches"] = sorted(slow_l, key=lambda x: -x["device_ms"])[:6]
        rep["slowest_renders"] = sorted(slow_r, key=lambda x: -x["device_ms"])[:4]
        rep["traces"] = len(traces)
        rep["requests"] = len(lat)
        rep["mpts_per_s"] = float(np.mean([x["mpts_per_s"] for x in reps]))
        rep["latency_ms"] = {"p50": float(np.percentile(lat, 50)),
                             "p99": float(np.percentile(lat, 99)),
                             "p99_per_trace": [x["latency_ms"]["p99"] for x in reps]}
        rep["admission_wait_ms"] = {"p50": float(np.percentile(wait, 50)),
                                    "p99": float(np.percentile(wait, 99))}
        out[name] = rep
    sv, pl = out["serving"], out["plain"]
    return {
        "workload": f"serving-16 octrees ({total} points, scale {args.serving_scale} of "
                    f"5M-200M points each)",
        "value": sv["mpts_per_s"], "unit": UNIT,
        "requests": len(reqs), "traces": len(traces), "request_points": "log-uniform 100k-5M",
        "arrival": f"Poisson, {rate / 1e6:.0f} Mpts/s (70% of the plain server's saturated "
                   f"throughput on the same trace, {cap / 1e6:.0f} Mpts/s)",
        "hbm_budget_bytes": budget,
        "frame": "1920x1080 render of every octree every 33.3 ms",
        "path": "serving form: HBM-budget admission, continuous batching, "
                "2 half-GPU persistent launches in flight",
        "inputs": "pinned host memory (copies inside the served latency)",
        "latency_ms": {"serving_p50": sv["latency_ms"]["p50"],
                       "serving_p99": sv["latency_ms"]["p99"],
                       "plain_p50": pl["latency_ms"]["p50"], "plain_p99": pl["latency_ms"]["p99"]},
        "serving": sv, "plain": pl, "saturated": sat,
        "h2d_bytes_per_trace": 16 * total, "gpu_launches": sv["launches"], "clocks": clk,
    }


def run_serving(args):
    """The serving form alone, as its own JSON line."""
    import torch

    from paper_2310_03567_gb300 import simlod
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    rank = int(os.environ.get("RANK", "0"))
    simlod.load()
    f = serving_form(args, rank)
    sv = f["serving"]
    line = {
        "metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 0, "ms_per_step": sv["seconds"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f["workload"], "requests": f["requests"],
                   "traces": f["traces"], "request_points": f["request_points"],
                   "arrival": f["arrival"], "hbm_budget_bytes": f["hbm_budget_bytes"],
                   "frame": f["frame"], "path": f["path"], "inputs": f["inputs"]},
        "latency_ms": f["latency_ms"], "serving": sv, "plain": f["plain"],
        "saturated": f["saturated"],
        "e2e": {"value": f["value"], "unit": UNIT,
                "h2d_bytes_per_step": f["h2d_bytes_per_trace"], "d2h_bytes_per_step": 0},
        "gpu_launches": f["gpu_launches"], "clocks": f["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_chunk_sweep(args):
    """Chunk-size study (the paper's chunk-size table, Section 7): the fused
    update of the workload and one 1080p frame for several points-per-chunk,
    with the data region each needs."""
    import torch

    from paper_2310_03567_gb300 import simlod
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    simlod.load()
    w, root_log2 = make_workload(args.workload, args.points, args.morton)
    dev_pts = simlod.points_tensor(w.points)
    ptrs = [dev_pts.data_ptr() + int(o) * 16 for o in w.offsets]
    counts = [int(c) for c in w.counts]
    side = float(1 << root_log2)
    ctr = np.asarray(w.root_min, float) + side * np.array([0.5, 0.5, 0.02])
    cam = simlod.view_proj(ctr + side * np.array([-0.45, -0.55, 0.35]), ctr, 60.0, 1920 / 1080)
    rows = []
    for C in (250, 500, 1000, 2000, 5000, 10000):
        tree = make_octree(w, root_log2, chunk_points=C)
        st_ = tree.stream
        for _ in range(args.warmup):
            tree.reset()
            if tree.insert_many_ptrs(ptrs, counts) != simlod.OK:
                raise RuntimeError("insert_batches")
        if tree.sync() != simlod.OK:
            raise RuntimeError(f"chunk {C}: update failed")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st_)
        for _ in range(args.steps):
            tree.reset()
            tree.insert_many_ptrs(ptrs, counts)
        e1.record(st_)
        torch.cuda.synchronize()
        if tree.sync() != simlod.OK:
            raise RuntimeError(f"chunk {C}: update failed")
        ms = e0.elapsed_time(e1) / args.steps
        st = tree.stats()
        frame = torch.empty((1080, 1920), dtype=torch.int64, device="cuda")
        tree.render(cam, frame)
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(st_)
        for _ in range(3):
            tree.render(cam, frame)
        r1.record(st_)
        torch.cuda.synchronize()
        payload = 20 * (st["points"] + st["voxels"])
        rows.append({"chunk_points": C, "mpts_per_s": w.n_points / ms / 1e3, "ms_per_step": ms,
                     "render_ms": r0.elapsed_time(r1) / 3, "data_used_bytes": st["data_used"],
                     "records_bytes": payload, "overhead": st["data_used"] / payload - 1.0,
                     "chunks": st["chunks_bumped"]})
        tree.close()
        del frame
        torch.cuda.empty_cache()
    base = next(r for r in rows if r["chunk_points"] == 1000)
    line = {"metric": METRIC, "value": base["mpts_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": w.name, "study": "points per chunk",
                                            "path": "fused persistent launch per step"},
            "chunk_sweep": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered",
                    choices=["aerial", "uniform", "clustered", "mixed", "serving"])
    ap.add_argument("--serving-traces", type=int, default=5,
                    help="independent Poisson traces whose requests the serving latency pools")
    ap.add_argument("--serving-scale", type=float, default=1.0,
                    help="octree sizes of the serving workload relative to 5M-200M points")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the batched and serving sub-measurements of the default run")
    ap.add_argument("--points", type=int, default=None)
    ap.add_argument("--batches", type=int, default=None,
                    help="only the first BATCHES batches of the workload (small profiling cases)")
    ap.add_argument("--ref-points", type=int, default=1_000_000,
                    help="reference arm: the first batches of the workload up to at least this "
                         "many points, per step")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chunk-sweep", action="store_true",
                    help="chunk-size study instead of the standard measurement")
    ap.add_argument("--morton", action="store_true",
                    help="sort the workload's stream in Morton order before cutting it")
    ap.add_argument("--max-batch", type=int, default=None,
                    help="octree batch capacity (staging) above the workload's largest batch: "
                         "lets the batched form merge small batches into larger updates")
    ap.add_argument("--batched", action="store_true",
                    help="also time the batched form (always on for --workload mixed)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.chunk_sweep:
        return run_chunk_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
