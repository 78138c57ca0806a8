"""Host-side arithmetic of bench.py that needs no GPU: the per-kind rate
table built from the library's live profile."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_rates_units_and_skips():
    names = {0: "gemm", 4: "mix", 8: "decide"}
    prof = {
        0: dict(ms=1200.0, launches=400, flops=2.4e15, bytes=0.0),     # 2 PFLOP over 1.2 s of 2 steps
        4: dict(ms=800.0, launches=200, flops=0.0, bytes=4.0e12),      # 4 TB over 0.8 s
        7: dict(ms=0.0, launches=0, flops=0.0, bytes=0.0),             # never ran: omitted
        8: dict(ms=50.0, launches=100, flops=0.0, bytes=0.0),          # timed only
    }
    r = bench.kernel_rates(prof, names, steps=2, hbm_gbs=8000.0)
    assert set(r) == {"gemm", "mix", "decide"}
    assert r["gemm"]["ms_per_step"] == 600.0 and r["gemm"]["launches_per_step"] == 200
    assert abs(r["gemm"]["gflops"] - 2.0e6) < 1e-6 and "gbs" not in r["gemm"]
    assert abs(r["mix"]["gbs"] - 5000.0) < 1e-9 and abs(r["mix"]["frac_hbm"] - 0.625) < 1e-12
    assert r["decide"] == {"ms_per_step": 25.0, "launches_per_step": 50.0}


def test_roofline_alu_peak_and_jacobi_traffic():
    """The FP32 Jacobi kind (1) is reported against the FP32 ALU peak of this
    device's SM count at the sampled clock, with its per-launch DRAM traffic
    scaled from the ncu capture by the launches' algorithmic bytes; the mix
    (4) against the measured copy bandwidth, with no traffic figure."""
    d = dict(ms=250.0, launches=400, flops=6.0e10, bytes=8.0e8)     # 2 MB of 8 r l a launch
    r = bench.roofline(d, 1, {"sm_mhz": 1000.0}, 100)
    peak = 100 * 128 * 2 * 1000.0e6 / 1e12
    assert r["bound"] == "alu" and abs(r["peak"] - peak) < 1e-12
    assert abs(r["achieved"] - 6.0e10 / 0.25 / 1e12) < 1e-12 and abs(r["frac"] - r["achieved"] / peak) < 1e-15
    assert abs(r["traffic"] - 0.635 * 2.0e6) < 1e-6 and "100 SMs" in r["peak_note"]
    assert r["launches"] == 400 and abs(r["avg_launch_us"] - 625.0) < 1e-9
    m = bench.roofline(dict(ms=100.0, launches=10, flops=0.0, bytes=5.0e11), 4, {"sm_mhz": 2070.0}, 152)
    hbm = bench.peaks()[0]
    assert m["bound"] == "hbm" and m["traffic"] is None
    assert abs(m["achieved"] - 5000.0) < 1e-9 and abs(m["frac"] - 5000.0 / hbm) < 1e-12
