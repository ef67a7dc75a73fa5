"""Host logic of bench.py, on the CPU: the traffic records' source-hash check,
the choice of the tensor peak, the clock-sample summary and the oracle baseline's
sampling (no GPU needed for any of these)."""
import hashlib
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_records_match_the_committed_sources():
    """Each record's kernel_source_sha256 is the hash of the listed sources as they
    stand; then recorded_traffic returns its bytes per launch."""
    for precision, (record, files) in bench.TRAFFIC_RECORDS.items():
        traffic, h = bench.recorded_traffic(files, record)
        m = hashlib.sha256()
        for f in files:
            with open(os.path.join(ROOT, f), "rb") as fh:
                m.update(fh.read())
        assert h == m.hexdigest()
        assert traffic is not None and traffic > 1e8, precision


def test_traffic_record_refused_for_changed_sources(tmp_path, monkeypatch):
    """A source that differs from the profiled one (one byte appended) voids the
    record: traffic None, so no stale figure is reported."""
    record, files = bench.TRAFFIC_RECORDS["fp64split"]
    root = tmp_path / "repo"
    for f in files + [record]:
        dst = root / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), dst)
    with open(root / files[0], "ab") as fh:
        fh.write(b"\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    traffic, _ = bench.recorded_traffic(files, record)
    assert traffic is None


def test_tensor_peak_burst_sustained_and_tf32():
    peaks = {"bf16_tflops": 1885.6, "bf16_tflops_sustained": 1689.9, "hbm_gbs": 6786.6}
    p, src = bench.tensor_peak(peaks, "measured", "fp64split", 1.0)
    assert p == 1885.6 and "bf16_tflops" in src and "sustained" not in src
    p, src = bench.tensor_peak(peaks, "measured", "bf16x6", 5.0)
    assert p == 1689.9 and "sustained" in src
    p, _ = bench.tensor_peak(peaks, "measured", "tf32x3", 1.0)
    assert p == pytest.approx(1885.6 * 1.1 / 2.25)
    for prec in ("fp64split40", "fp64split32"):  # BF16 slice products
        assert bench.tensor_peak(peaks, "measured", prec, 1.0)[0] == 1885.6


def test_clock_summary_reads_reasons_and_median():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler(0).summary() is None


def test_cpu_baseline_compares_then_extends_the_sample():
    """The oracle runs the GPU's step count (the compared field), then further
    timed steps up to max_steps; with no GPU field nothing is compared."""
    out = bench.cpu_baseline("ac2d_64", None, 5, max_steps=20, min_seconds=60.0)
    assert out["kind"] == "oracle" and out["cores"] >= 1
    assert out["sample"].startswith("20 FP64 time steps") and "the first 5 compared" in out["sample"]
    assert "rel_err_vs_gpu" not in out
    assert out["value"] > 0
