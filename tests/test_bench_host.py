"""Host-side logic of the benchmark (CPU): the DRAM traffic of the roofline is
reported only for the captured kernel variant and workload and only while the
kernel's source section still hashes to the captured one; the filter-active
eps comes from the norm products' percentile."""
import importlib
import os
import shutil

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    import sys

    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_traffic_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    """The stored DRAM traffic is reported while every code section that
    decides it (the kernel, the row-order work list, the host order) is
    unchanged, and dropped when any of them changes."""
    bench = _bench()
    entry = dict(bench.MEASURED_TRAFFIC[("pk12", "water2048")])
    for src, _, _ in entry["sections"]:
        (tmp_path / os.path.dirname(src)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), tmp_path / src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry["sections"] = [(src, sec, bench.kernel_source_sha(src, sec)) for src, sec, _ in entry["sections"]]
    assert all(sha is not None for _, _, sha in entry["sections"])
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, ("pk12", "water2048"), entry)
    assert bench.measured_traffic("pk12", "water2048") == entry["bytes"]
    assert bench.measured_traffic("pk16", "water2048") is None
    assert bench.measured_traffic("pk12", "amorphous4096") is None
    # one section changes: the captured counters no longer describe the code
    for src, sec, _ in entry["sections"]:
        text = (tmp_path / src).read_text()
        a = text.index(sec[0]) + len(sec[0])
        (tmp_path / src).write_text(text[:a] + "// edited\n" + text[a:])
        assert bench.measured_traffic("pk12", "water2048") is None
        (tmp_path / src).write_text(text)
        assert bench.measured_traffic("pk12", "water2048") == entry["bytes"]


def test_eps_percentile_of_norm_products():
    bench = _bench()
    A = synth.water(8, seed=2)
    eps = bench.norm_product_percentile(A, 30)
    assert eps > 0 and np.isfinite(eps)
    # a higher percentile gives a larger threshold
    assert bench.norm_product_percentile(A, 60) > eps


def test_fp64_peak_derived_from_sms_and_clock():
    bench = _bench()
    peak, src = bench.fp64_peak_gflops(152, {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0})
    assert abs(peak - 152 * 4 * 2.070) < 1e-9 and "derived" in src
    # a lower sampled clock lowers the peak in proportion
    low, _ = bench.fp64_peak_gflops(152, {"sm_mhz": 1035.0, "sm_max_mhz": 2070.0})
    assert abs(low - peak / 2) < 1e-9
    # no samples: the maximum clock
    nos, src2 = bench.fp64_peak_gflops(152, {"sm_mhz": None, "sm_max_mhz": None})
    assert nos > 0 and "no clock samples" in src2
