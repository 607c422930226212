"""The benchmark's roofline bookkeeping, on the CPU (no GPU needed).

* achieved = the method's flop for one sigma build of the main exchange
  contraction, 2 M N K with M = 2T nocc, N = nvirt, K = naux nvirt (one
  product, whatever the precision's hi/lo split), divided by the class's
  time per sigma build;
* a tensor-bound class is set against the sustained bf16 peak, with the
  burst fraction beside it;
* the DRAM traffic comes from the committed ncu table only for exactly the
  workload, precision and plan it was captured with, and never for a
  chunked exchange.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.set_workload("fieldscan")
    return b


PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1700.0, "bf16_tflops_sustained": 1400.0}
PLAN = {"main_kernel": 2, "main_bn": 192, "main_mb": 2, "main_kb": 64, "main_splits": 8, "z_chunk": 3072,
        "main_cluster": 4, "main_grid": 132}


def test_main_contraction_counts_one_product_against_the_sustained_peak(bench):
    T, nsig, ms_per_sigma = 32, 40, 21.0
    o, v, P = 128, 768, 3072
    flop = 2.0 * (2 * T * o) * v * (P * v)
    for prec, nprod in (("bf16", 1), ("bf16x2", 2)):
        r = bench.roofline(prec, "exchange_main", (ms_per_sigma * nsig, nsig), T, PEAKS, nsig, PLAN)
        assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
        assert r["flop_per_sigma"] == pytest.approx(flop)
        assert r["achieved"] == pytest.approx(flop / (ms_per_sigma / 1e3) / 1e12)
        assert r["peak"] == PEAKS["bf16_tflops_sustained"]
        assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["bf16_tflops_sustained"])
        assert r["frac_of_burst"] == pytest.approx(r["achieved"] / PEAKS["bf16_tflops"])
        assert r["hardware_tflops"] == pytest.approx(nprod * r["achieved"])


def _table_bytes(cls):
    """Bytes per sigma of the committed ncu table's row for the field scan's
    plain-BF16 plan and kernel class."""
    want = ["fieldscan", "3072", "bf16", cls] + [str(PLAN[k]) for k in (
        "main_kernel", "main_bn", "main_mb", "main_kb", "main_splits", "main_cluster", "main_grid")]
    for line in open(os.path.join(ROOT, "profiles", "dram_traffic.txt")):
        f = line.split("#", 1)[0].split()
        if f[:11] == want:
            return float(f[11])
    raise AssertionError(f"no row for {cls}")


def test_traffic_only_for_the_captured_plan(bench):
    z = bench.roofline("bf16", "exchange_z", (10.0 * 40, 80), 32, PEAKS, 40, PLAN)
    assert z["bound"] == "hbm" and z["unit"] == "GB/s"
    assert z["traffic"] == pytest.approx(_table_bytes("exchange_z"))
    assert z["traffic_over_algorithmic"] == pytest.approx(z["traffic"] / z["bytes_per_sigma"])
    # the Z build writes the 38.65 GB of Z and reads B_oo: its traffic is close to its algorithmic bytes
    assert 0.99 < z["traffic_over_algorithmic"] < 1.1
    m = bench.roofline("bf16", "exchange_main", (21.0 * 40, 40), 32, PEAKS, 40, PLAN)
    assert m["traffic"] == pytest.approx(_table_bytes("exchange_main"))
    for change in ({"main_cluster": 1}, {"main_grid": 148}, {"main_splits": 9}, {"main_kb": 32},
                   {"z_chunk": 512}):
        other = dict(PLAN, **change)
        assert bench.roofline("bf16", "exchange_main", (21.0 * 40, 40), 32, PEAKS, 40, other)["traffic"] is None
    assert bench.roofline("bf16x2", "exchange_main", (21.0 * 40, 40), 32, PEAKS, 40, PLAN)["traffic"] is None
