"""Host-side arithmetic of the bench line, on the CPU: the algorithmic bytes
behind the roofline fractions (the 20-byte records with gidx, and the
paper's 16-byte records) and the host description beside the CPU oracle."""
import bench


def test_algorithmic_bytes_per_update():
    # 16 B read + 20 B written per point, 40 B per re-inserted point, 16 B per
    # voxel, one zeroed grid per split
    assert bench.update_alg_bytes(10, 0, 0, 0, 262_144) == 360
    assert bench.update_alg_bytes(0, 3, 0, 0, 262_144) == 120
    assert bench.update_alg_bytes(0, 0, 5, 0, 262_144) == 80
    assert bench.update_alg_bytes(0, 0, 0, 2, 262_144) == 524_288


def test_paper_style_roofline_counts_16_byte_records():
    B, S, V, K, grid = 1_000_000, 200_000, 300_000, 4, 262_144
    r = bench.paper_style_roofline(B, S, V, K, grid, peak_gbs=1000.0, mpts=100.0)
    b = 32 * B + 32 * S + 16 * V + grid * K
    assert r["alg_bytes_per_point"] == b / B
    # the roofline: points per second at which b bytes take the peak's time
    assert abs(r["roofline_mpts"] - B / (b / 1e12) / 1e6) < 1e-6
    assert abs(r["frac"] - 100.0 / r["roofline_mpts"]) < 1e-12
    # fewer bytes per point than the gidx-carrying figure, so a higher roofline
    full = bench.update_alg_bytes(B, S, V, K, grid)
    assert b < full


def test_host_cpu_names_the_cores():
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and h["model"] and h["arch"]
