"""bench.py's host-side arithmetic on the CPU: the oracle's whole-step
extrapolation from timed calls, and the CPU description it records."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_oracle_extrapolation_counts_weights_once_per_call():
    import bench
    from paper_1404_3458_gb300 import workloads as WL

    w = WL.WORKLOADS["large_gf16"]
    rows = 64
    # calls evaluating `rows` rows cost the weights plus rows x per-row cost
    t_we, t_wd, per_e, per_d = 8.0, 9.0, 0.1, 0.08
    step, pe, pd = bench.oracle_extrapolate(w, rows, t_we, t_wd, t_we + rows * per_e, t_wd + rows * per_d)
    assert pe == pytest.approx(per_e) and pd == pytest.approx(per_d)
    assert step == pytest.approx(t_we + (w.n - w.k) * per_e + t_wd + w.erasures * per_d)
    # a noisy sample whose row calls came out faster than the weights alone
    # never gives a negative per-row cost
    step2, pe2, _ = bench.oracle_extrapolate(w, rows, 8.0, 8.0, 7.9, 8.5)
    assert pe2 == 0.0 and step2 > 16.0


def test_host_cpu_reports_model_and_cores():
    import bench

    cpu = bench.host_cpu()
    assert cpu["nproc"] == os.cpu_count() and cpu["machine"] and cpu["model"]
