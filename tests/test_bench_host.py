"""Host-side logic of bench.py (CPU): algorithmic bytes per layout, the
clock-sample summary that decides whether a run is valid, and the reference
arm naming the same workload as the arm it stands beside."""
import pytest

import bench


@pytest.mark.parametrize("dim,layout,coupled,per_node", [
    # 2D lattice: u 16+16, v 16+16, a 8+8, 1/m 4, bond word 4, + body 8 | alpha 4 + g 8
    (2, 1, False, 96), (2, 1, True, 100),
    # 3D lattice: u 24+24, v 24+24, a 16+16, 1/m 4, four bond words 16, + body 12 | alpha 4 + g 12
    (3, 2, False, 160), (3, 2, True, 164),
])
def test_algorithmic_bytes_per_node(dim, layout, coupled, per_node):
    n, nb = 1000, 28000
    info = {"dim": dim, "layout": layout, "n": n, "n_bonds": nb}
    total, node = bench.algorithmic_bytes(info, None, with_body=not coupled, coupled=coupled)
    assert node == per_node and total == per_node * n


def test_sliced_ell_bytes_count_the_family_list():
    info = {"dim": 2, "layout": 0, "n": 1000, "n_bonds": 28000}
    total, node = bench.algorithmic_bytes(info, None, with_body=True, coupled=False)
    # 4 B family word and one status bit per directed bond, plus the node state
    assert node == 92 and total == 4 * 28000 + 28000 / 8 + 92 * 1000


def test_clock_summary_reports_throttle_reasons():
    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.samples = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["0", "1980", "2070", "1390", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
                 ["0", "2070", "2070", "1000", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.samples.append(["0", "1500", "2070", "1000", "0x8", "Active", "Not Active", "Not Active", "Not Active"])
    assert "hw_slowdown" in c.summary()["reasons"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_reference_arm_names_the_arm_workload():
    assert bench.reference_problem("coupled")[0] == bench.COUPLED_NAME
    assert bench.reference_problem("coupled3d")[0] == bench.COUPLED3D_NAME
    assert bench.reference_problem("pd")[0] == bench.WORKLOAD["name"]
    assert bench.reference_problem("batch")[0] == bench.BATCH_NAME.format(n=64)
    # the coupled plate's PD lattice is the 800,000-node strip the arm advances
    assert bench.reference_problem("coupled")[1].n == 2000 * 400


def test_issue_and_l2_lines():
    """The issue-rate line puts ncu's warp instructions per launch over the
    live launch time against 152 SMs x 4 schedulers x the sampled clock; the
    L2 line puts the SMs' L2 bytes per launch against the stored nominal rate.
    Without stored counts both lines carry the peak and no fraction."""
    ent = {"warp_instructions_per_launch": 12_000_000, "l2_bytes_per_launch": 120_000_000}
    issue, l2 = bench.issue_and_l2(ent, 0.02, {"sm_mhz": 2000.0}, 152, 36000.0)
    assert issue["peak"] == 152 * 4 * 2000e6
    assert issue["achieved"] == pytest.approx(12e6 / 20e-6)
    assert issue["frac"] == pytest.approx(6e11 / 1.216e12)
    assert l2["achieved"] == pytest.approx(120e6 / 20e-6 / 1e9)
    assert l2["frac"] == pytest.approx(6000.0 / 36000.0)
    issue, l2 = bench.issue_and_l2({}, 0.02, {"sm_mhz": None}, 152, None)
    assert issue["peak"] == 152 * 4 * 2070e6 and issue["frac"] is None and l2["frac"] is None


def test_stored_counters_follow_the_kernel_source():
    """profiles/traffic.json's figures are reported only under the hash of the
    kernel source they were measured on (2D and 3D hashed separately)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")) as f:
        tj = json.load(f)
    for wl, tiles in tj.items():
        if not isinstance(tiles, dict):
            continue
        for tile, ent in tiles.items():
            got, peak = bench.stored_counters(wl, tile)
            assert peak == tj["l2_peak_gbs"]
            assert (got == ent) == (ent["kernel_version"] == bench.kernel_version(wl))
    assert bench.kernel_version("coupled") == bench.kernel_version("pd") != bench.kernel_version("coupled3d")
