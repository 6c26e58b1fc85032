"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/simlod.h declares. Host-only calls (no CUDA work) are exercised;
nothing here needs a GPU."""
import ctypes
import os
import re

import pytest

from paper_2310_03567_gb300 import _build, simlod

HEADER = os.path.join(_build.INCLUDE_DIR, "simlod.h")


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"SIMLOD_API\s+[\w\s\*]+?\b(simlod_\w+)\s*\(", text)


@pytest.fixture(scope="module")
def lib():
    _build.build_library()
    return simlod.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("simlod_create", "simlod_insert_batch", "simlod_snapshot", "simlod_destroy"):
        assert required in names
    assert len(names) == len(set(names))


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in simlod.SIGNATURES, f"binding lacks {name}"


def test_library_is_sm103a_only():
    cmds = [c for c, _ in _build.compile_commands()] + [_build.link_command(["x.o"], "x.so")]
    for cmd in cmds:
        assert "arch=compute_103a,code=sm_103a" in cmd
        assert sum(1 for a in cmd if a == "-gencode") == 1
    # every kernel instance of the autotuner is built, each in its own namespace
    assert len(cmds) == len(_build.library_sources()) + len(_build.VARIANTS) + 1
    assert len({a for c in cmds for a in c if a.startswith("-DSL_NS=")}) == len(_build.VARIANTS)


def test_no_oracle_on_the_product_path():
    pkg = os.path.dirname(_build.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                src = open(os.path.join(root, f), errors="replace").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "oracle.h" not in src, f


def test_config_default_is_the_papers(lib):
    cfg = simlod.default_config()
    assert cfg.leaf_capacity == 50_000      # Section 3.1
    assert cfg.chunk_points == 1_000        # Section 3.4
    assert cfg.grid_log2 == 7               # 128^3, Section 3.3
    assert cfg.backlog_capacity == 10_000_000  # Section 5.2


def test_struct_sizes_match_header(lib):
    assert ctypes.sizeof(simlod.Config) == 4 * 3 + 4 * 5 + 8 * 4 + 8
    assert simlod.NODE_DTYPE.itemsize == ctypes.sizeof(simlod.NodeRec) == 48
    assert simlod.POINT_REC_DTYPE.itemsize == 20 and simlod.VOXEL_REC_DTYPE.itemsize == 20


def test_arena_bytes_and_invalid_configs(lib):
    cfg = simlod.default_config()
    a = simlod.arena_bytes(cfg, 1 << 30)
    assert a > (1 << 30)
    for bad in (dict(root_log2=0), dict(root_log2=32), dict(grid_log2=8), dict(chunk_points=0),
                dict(leaf_capacity=0), dict(max_nodes=4), dict(max_nodes=(1 << 27) + 1),
                dict(backlog_capacity=0)):
        c = simlod.default_config(**bad)
        out = ctypes.c_uint64()
        assert lib.simlod_arena_bytes(ctypes.byref(c), 1 << 20, ctypes.byref(out)) == \
            simlod.ERR_INVALID_ARG, bad
    # the largest node table (mover entries pack a node id into 27 bits)
    c = simlod.default_config(max_nodes=1 << 27)
    out = ctypes.c_uint64()
    assert lib.simlod_arena_bytes(ctypes.byref(c), 1 << 30, ctypes.byref(out)) == simlod.OK
    # a root cube running past int32 is invalid
    c = simlod.default_config(root_min=(2**31 - 10, 0, 0), root_log2=10)
    out = ctypes.c_uint64()
    assert lib.simlod_arena_bytes(ctypes.byref(c), 0, ctypes.byref(out)) == simlod.ERR_INVALID_ARG


def test_create_rejects_bad_arguments_before_cuda(lib):
    cfg = simlod.default_config()
    h = ctypes.c_void_p()
    # null arena, misaligned arena, bad config: all rejected before any CUDA call
    assert lib.simlod_create(ctypes.byref(cfg), None, 1 << 30, None, ctypes.byref(h)) == \
        simlod.ERR_INVALID_ARG
    assert lib.simlod_create(ctypes.byref(cfg), 0x1001, 1 << 30, None, ctypes.byref(h)) == \
        simlod.ERR_INVALID_ARG
    bad = simlod.default_config(grid_log2=9)
    assert lib.simlod_create(ctypes.byref(bad), 0x100000, 1 << 30, None, ctypes.byref(h)) == \
        simlod.ERR_INVALID_ARG
    assert lib.simlod_insert_batch(None, None, 0, None) == simlod.ERR_INVALID_ARG
    assert lib.simlod_destroy(None) == simlod.ERR_INVALID_ARG


def test_null_handles_are_rejected_before_cuda(lib):
    """Every entry point that takes a handle or a plan refuses a null one with
    INVALID_ARG, touching nothing (this machine has no GPU)."""
    calls = {
        "simlod_insert_batch_host": (None, None, 0, None),
        "simlod_insert_batches": (None, None, None, 0, None),
        "simlod_insert_batches_budget": (None, None, None, 0, 0, None),
        "simlod_progress": (None, None, None),
        "simlod_insert_batches_host": (None, None, None, 0, None, None, None, None),
        "simlod_plan_create": (None, None, None, 0, None, None),
        "simlod_plan_run": (None, None),
        "simlod_plan_info": (None, None, None),
        "simlod_plan_destroy": (None,),
        "simlod_plan_autotune": (None, None, None, 0, None, None, None),
        "simlod_set_launch_width": (None, 1, None),
        "simlod_frame_update": (None, None, None, 0, 0, None, None),
        "simlod_reset": (None, None),
        "simlod_sync": (None,),
        "simlod_get_stats": (None, None),
        "simlod_snapshot": (None, None),
        "simlod_render": (None, None, 1, 1, None, 0, None),
        "simlod_restore": (None, None, None),
        "simlod_set_timing": (None, 1, 0),
        "simlod_get_timing": (None, None),
        "simlod_set_wait_limits": (None, 0, 0),
        "simlod_compact": (None, 0, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == simlod.ERR_INVALID_ARG, name


def test_status_strings(lib):
    for code in range(-11, 1):
        s = simlod.status_string(code)
        assert s and s != "unknown status"
    assert simlod.status_string(-99) == "unknown status"


def test_kernel_instance_count_agrees(lib):
    text = open(HEADER).read()
    n = int(re.search(r"#define SIMLOD_N_VARIANTS (\d+)", text).group(1))
    internal = open(os.path.join(_build.CSRC_DIR, "variant.h")).read()
    assert int(re.search(r"#define SL_N_VARIANTS (\d+)", internal).group(1)) == n
    assert simlod.N_VARIANTS == n == len(_build.VARIANTS) + 1
    d = simlod.VariantDesc()
    assert lib.simlod_variant_info(n, ctypes.byref(d)) == simlod.ERR_INVALID_ARG
    assert lib.simlod_variant_info(0, None) == simlod.ERR_INVALID_ARG
