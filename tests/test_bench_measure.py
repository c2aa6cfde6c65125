"""The benchmark's roofline arithmetic on hand-computed cases (no GPU): the plain-ALU peak
and the method's algorithmic bytes per stage and per timed kernel."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_alu_peak_is_lanes_times_clock():
    # 152 SMs x 128 lanes x 2070 MHz, one 32-bit operation per lane per clock
    assert math.isclose(bench.alu_peak_tops(152, 2070.0), 40.27392, rel_tol=1e-12)
    assert math.isclose(bench.alu_peak_tops(1, 1000.0), 0.128, rel_tol=1e-12)


def test_algorithmic_bytes_by_hand():
    # three halos: 100 members (below N_search, not searched, at most N_se: small f_l),
    # 200 members (searched, small f_l) and 1000 members (searched, big f_l)
    sizes = [100, 200, 1000]
    n = 5000
    stage, kern = bench.algorithmic_bytes(n, sizes, nse=256, nsearch_min=160)
    assert stage["fof3d"] == 16.0 * n
    assert stage["velden"] == 32.0 * 1300
    assert stage["outlier_ratio"] == 40.0 * 1200 and stage["fof6d"] == 32.0 * 1200
    # N_cell: max(0.01 N_H, min(100, N_H / 8)) -> 25 and 100 members per leaf; tree levels
    # ceil(log2(N_H / N_cell)) = 3 and 4
    assert bench.ncell_rule(200) == 25 and bench.ncell_rule(1000) == 100
    cells = (16.0 * 3 + 24.0) * 200 + (16.0 * 4 + 24.0) * 1000
    assert stage["cells"] == cells
    assert kern["velden_big"] == 32.0 * 1000 and kern["velden_small"] == 32.0 * 300
    assert kern["cells_build"] + kern["cells_build_big"] == cells and kern["cells_build_big"] == 0
    assert kern["ell_fit"] == 8.0 * 1200 and kern["ratio"] == 40.0 * 1200
    assert kern["fof_link"] == 16.0 * n and kern["halo_frame"] == 12.0 * 1300
