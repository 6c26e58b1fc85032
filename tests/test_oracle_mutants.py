"""The oracle's pins catch plausible mistakes.

Each case copies the oracle sources, plants one mistake (a wrong threshold,
a transposed index, a dropped term, a changed order), builds the copy and
runs the quick pins against it in a child process: every mutant must fail.
The mistakes are planted only in throw-away copies of the oracle on the CPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    "split_at_T": ("incremental.c", "nd->counter > T && nd->log2size > 0",
                   "nd->counter >= T && nd->log2size > 0"),
    "counter_starts_at_zero": ("incremental.c", "nd->counter = nd->num_points;",
                               "nd->counter = 0;"),
    "octant_axes_swapped": ("incremental.c", "return bx | (by << 1) | (bz << 2);",
                            "return by | (bx << 1) | (bz << 2);"),
    "cell_axes_swapped": ("incremental.c", "return c[0] + (c[1] << G) + (c[2] << (2 * G));",
                          "return c[1] + (c[0] << G) + (c[2] << (2 * G));"),
    "centre_drops_half": ("incremental.c", "(uint64_t)(2 * c[a] + 1)", "(uint64_t)(2 * c[a])"),
    "batch_sampled_before_spill": ("incremental.c",
                                   "int from_spill = k < spill.n;",
                                   "int from_spill = k >= n;"),
    "stop_descent_after_claim": ("incremental.c", "        nd->vox_counter++;\n",
                                 "        nd->vox_counter++;\n        break;\n"),
    "spill_not_recounted": ("incremental.c", "      if (!leaf->final) leaf->counter++;\n    }\n    /* Splitting",
                            "      (void)leaf;\n    }\n    /* Splitting"),
    "chunk_count_off_by_one": ("incremental.c", "uint64_t need = (total + C - 1) / C;",
                               "uint64_t need = total / C + 1;"),
    "static_split_at_T": ("static.c", "if (!(n > t->cfg.leaf_capacity && L > 0))",
                          "if (!(n >= t->cfg.leaf_capacity && L > 0))"),
    "static_last_point_wins": ("static.c", "    if (bc->seen[cell]) continue;\n",
                               "    if (bc->seen[cell]) { t->voxels[t->n_voxels - 1].rgba = rgba_of(p); continue; }\n"),
    "static_child_min_swapped": ("static.c", "int32_t cm[3] = {(int32_t)(mn[0] + ((o & 1) ? half : 0)), (int32_t)(mn[1] + ((o & 2) ? half : 0)),",
                                 "int32_t cm[3] = {(int32_t)(mn[0] + ((o & 2) ? half : 0)), (int32_t)(mn[1] + ((o & 1) ? half : 0)),"),
    # renderer (Section 6)
    "render_lod_half_threshold": ("render.c", "const float lod = (float)(1u << r->cfg->grid_log2);",
                                  "const float lod = (float)(1u << (r->cfg->grid_log2 - 1));"),
    "render_depth_from_x": ("render.c", "memcpy(&depth, &c.cw, 4);", "memcpy(&depth, &c.cx, 4);"),
    "render_pixel_rounded": ("render.c", "const uint32_t px = (uint32_t)sx, py = (uint32_t)sy;",
                             "const uint32_t px = (uint32_t)(sx + 0.5f), py = (uint32_t)(sy + 0.5f);"),
    "render_cull_any_corner": ("render.c", "*culled = out[0] == 8 || out[1] == 8 || out[2] == 8 || out[3] == 8 || out[4] == 8;",
                               "*culled = out[0] > 0 || out[1] == 8 || out[2] == 8 || out[3] == 8 || out[4] == 8;"),
    "render_farthest_wins": ("render.c", "if (key < *f) *f = key;", "if (key > *f || *f == ~0ull) *f = key;"),
    "render_height_uses_width": ("render.c", "const float sx = screen(c.cx, c.cw, (float)W), sy = screen(c.cy, c.cw, (float)H);",
                                 "const float sx = screen(c.cx, c.cw, (float)W), sy = screen(c.cy, c.cw, (float)W);"),
    "render_parent_also_drawn": ("render.c", "  if (!n->is_inner || !(size > lod)) {\n    draw_node(r, k);\n    return;\n  }",
                                 "  draw_node(r, k);\n  if (!n->is_inner || !(size > lod)) return;"),
}

SOURCES = ("incremental.c", "static.c", "render.c")
PINS = {
    "incremental.c": ("test_oracle.py", "worked_example or brute_force_tiny or offset_root or "
                      "partition_independence or unsplittable or prefixes"),
    "static.c": ("test_oracle.py", "worked_example or brute_force_tiny or offset_root or "
                 "partition_independence or unsplittable or prefixes"),
    "render.c": ("test_oracle_render.py", ""),
}


def build_copy(tmp_path, fname=None, old=None, new=None):
    for f in SOURCES + ("oracle.h",):
        shutil.copy(os.path.join(ORACLE, f), tmp_path / f)
    if fname:
        src = (tmp_path / fname).read_text()
        assert src.count(old) == 1, f"mutation anchor not found once in {fname}: {old!r}"
        (tmp_path / fname).write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_copy.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    *[str(tmp_path / f) for f in SOURCES], "-o", str(lib), "-lm"], check=True)
    return lib


def run_pins(lib, test_file, select):
    env = dict(os.environ, SIMLOD_ORACLE_LIB=str(lib))
    tests = os.path.join(os.path.dirname(os.path.abspath(__file__)), test_file)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", tests]
    if select:
        cmd += ["-k", select]
    return subprocess.run(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                          text=True, timeout=600)


@pytest.mark.parametrize("test_file", ["test_oracle.py", "test_oracle_render.py"])
def test_unmodified_copy_passes_the_pins(test_file, tmp_path):
    """Control: the copy without a planted mistake passes the same pins, so a
    mutant fails because of its mistake."""
    lib = build_copy(tmp_path)
    select = PINS["incremental.c" if test_file == "test_oracle.py" else "render.c"][1]
    proc = run_pins(lib, test_file, select)
    assert proc.returncode == 0, proc.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    fname, old, new = MUTANTS[name]
    lib = build_copy(tmp_path, fname, old, new)
    test_file, select = PINS[fname]
    proc = run_pins(lib, test_file, select)
    assert proc.returncode != 0, f"mutant {name} survived the pins:\n{proc.stdout[-2000:]}"
