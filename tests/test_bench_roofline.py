"""bench.py's roofline object on CPU: the dominant kernel's algorithmic rate
(4 flops per visibility-pixel pair per operator pass) against the measured
burst bf16 peak, the 3-term split's executed rate and cap, and the traffic
record only for the workload it was captured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_roofline_of_the_dominant_tensor_kernel():
    import bench
    peaks, src = bench._peaks()
    units = 999600 * 256 * 256
    kprof = {"fwd_tc": (4.81, 10), "adj_tc": (4.45, 10), "prep": (0.14, 10), "adj_reduce_grad": (0.18, 10)}
    r = bench.roofline(kprof, units, 2)
    achieved = 4.0 * units / 0.481e-3 / 1e12
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(achieved)
    assert r["peak"] == peaks["bf16_tflops"]
    assert r["frac"] == pytest.approx(achieved / peaks["bf16_tflops"])
    assert r["executed_frac"] == pytest.approx(3 * r["frac"])
    assert r["algorithmic_cap"] == pytest.approx(1 / 3)
    assert r["note"].startswith("fwd_tc: 0.481 ms/launch")
    assert r["traffic"] == bench._traffic("fwd_tc")
    # another workload: the committed traffic record does not apply
    assert bench.roofline(kprof, units, 5)["traffic"] is None
    # the adjoint dominant
    r = bench.roofline({"fwd_tc": (4.0, 10), "adj_tc": (4.5, 10)}, units, 2)
    assert r["note"].startswith("adj_tc: 0.450 ms/launch")
    assert r["traffic"] == bench._traffic("adj_tc")


def test_traffic_record_is_current_for_the_committed_sources():
    # the record is valid only while the hash of the kernel sources matches;
    # a stale record must read as None (the bench then reports no traffic)
    import bench
    for k in ("fwd_tc", "adj_tc"):
        t = bench._traffic(k)
        assert t is None or 20e6 < t < 60e6


def test_roofline_of_the_fp32_direct_form_is_against_the_sfu():
    import bench
    units = 999600 * 256 * 256
    r = bench.roofline({"fwd_direct_f32": (270.0, 10), "adj_direct_f32": (440.0, 10)}, units, 2)
    assert r["bound"] == "alu" and r["unit"].startswith("Top/s")
    assert r["achieved"] == pytest.approx(2.0 * units / 44.0e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 16 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
