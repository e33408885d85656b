"""Host-side helpers of bench.py (no GPU): the clock summary read from nvidia-smi samples,
the measured HBM peak, and the algorithmic flop count of the cell apply quoted in the
roofline (260,580 flop per cell and vector at p = 6, n_q = 8, k != 0)."""
import json
import os

import bench


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_median_and_reasons(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    with open(cs.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    cs.proc = _Done()
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_hbm_peak_reads_the_measured_file():
    peak, note = bench.hbm_peak()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert peak == json.load(open(path))["hbm_gbs"] and "measured" in note
    else:
        assert peak == 6800.0 and "fallback" in note


def test_cell_apply_flop_count():
    assert bench.flops_per_cell_vector(6, 8, True) == 260580
    assert bench.flops_per_cell_vector(6, 8, False) < 260580      # no -i k.grad terms at k = 0


def test_cell_traffic_scales_the_captured_variants_only():
    """roofline.traffic: the DRAM bytes of a captured variant at 32 vectors, the 34 MB of fields
    fixed and the rest scaled by the vector count; null (with a reason) for a variant that has
    no capture of the current kernel."""
    for var, per32 in bench.CELL_TRAFFIC_32.items():
        t32, _ = bench.CELL_TRAFFIC(32, var)
        t256, note = bench.CELL_TRAFFIC(256, var)
        assert abs(t32 - per32) < 1.0
        assert abs(t256 - (0.034e9 + (per32 - 0.034e9) * 8)) < 1.0 and str(var) in note
    assert 4 in bench.CELL_TRAFFIC_32             # the variant the tuner picks at p = 6, 256 vectors
    t, note = bench.CELL_TRAFFIC(256, 0)
    assert t is None and "no ncu capture" in note
