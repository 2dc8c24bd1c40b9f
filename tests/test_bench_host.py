"""Host-side logic of bench.py (CPU only): the roofline denominators, the
per-launch DRAM traffic that is reported only while the profiled kernel
sources are unchanged, and the replica throughput."""
import hashlib
import json
import os
import shutil

import pytest

import bench


def _copy_tree_for(key, tmp_path):
    """A copy of profiles/traffic.json and of the sources one entry hashes."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    for f in d[key]["sources"]:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, f), dst)
    return d[key]


def test_every_traffic_entry_names_existing_sources_and_profile():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    assert d
    for key, e in d.items():
        assert e["bytes_per_launch"] > 0, key
        for f in e["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, f)), (key, f)
        prof = e["from"].split(":")[0]
        assert prof.startswith("profiles/") and os.path.exists(os.path.join(bench.ROOT, prof)), (key, prof)
        assert len(e["source_sha256"]) == 64


@pytest.mark.parametrize("key", ["k1pp_f32x2_n1024", "k1pp_bf16_n1024"])
def test_traffic_is_dropped_once_a_source_changes(key, tmp_path, monkeypatch):
    e = _copy_tree_for(key, tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = hashlib.sha256()
    for f in e["sources"]:
        h.update((tmp_path / f).read_bytes())
    expect = e["bytes_per_launch"] if h.hexdigest() == e["source_sha256"] else None
    assert bench.kernel_traffic(key) == expect
    # one byte more in any source: the counters no longer describe the kernel
    last = tmp_path / e["sources"][-1]
    last.write_bytes(last.read_bytes() + b"\n")
    assert bench.kernel_traffic(key) is None
    assert bench.kernel_traffic("no_such_kernel") is None


def test_headline_traffic_matches_the_current_sources():
    # the bench line's traffic of its default workload (the F32X2 persistent
    # stepper at N = 1024) describes the kernel as it is now
    assert bench.kernel_traffic("k1pp_f32x2_n1024") is not None


def test_traffic_absent_without_summary(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k1pp_bf16_n1024") is None


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, 1900.0, 1700.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5, "bf16_tflops": 2000}))
    assert bench.peaks() == (7000.5, 2000.0, 0.0, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text(
        json.dumps({"hbm_gbs": 6782.1, "bf16_tflops": 1918.6, "bf16_tflops_sustained": 1726.0}))
    assert bench.peaks() == (6782.1, 1918.6, 1726.0, "measured")


def test_replica_throughput_counts_every_replica():
    assert bench.replica_throughput(0.5, 1) == pytest.approx(2000.0)
    assert bench.replica_throughput(0.5, 8) == pytest.approx(16000.0)


def test_reference_arm_prints_one_contract_line():
    # the oracle arm of the bench on the host cores, at a small N
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and d["dtype"] == "f64"
