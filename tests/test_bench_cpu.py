"""Host-side pieces of bench.py (no GPU): the reference arm's JSON line, the
reading of the committed ncu summaries and of the measured peaks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CONTRACT_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--side", "512", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert CONTRACT_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_are_silent():
    env = dict(os.environ, RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--side", "512", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_profile_summary_fields_parse():
    """The streaming-kernel summary names its source hash; when that is the
    current one, the fields the bench line uses read as numbers."""
    path = os.path.join(ROOT, "profiles", "fused_extract_16384_u16.txt")
    kv = dict(ln.split(":", 1) for ln in open(path) if ":" in ln and not ln.startswith("#"))
    assert len(kv["source_sha256"].strip()) == 64
    if kv["source_sha256"].strip() != bench.kernel_source_sha():
        pytest.skip("kernel sources changed since the summary was captured (the bench reports null)")
    lane = bench.profiled("fused_extract_16384_u16", "lane_inst_per_px")
    traffic = bench.profiled_traffic("fused_extract_16384_u16")
    assert 20 < lane < 1000
    # within a factor of two of the algorithmic 3 B/px of a 16384^2 launch
    assert 0.5 * 3 * 16384 ** 2 < traffic < 2 * 3 * 16384 ** 2


def test_profiled_is_none_for_unknown_kernel_or_field():
    assert bench.profiled("no_such_kernel", "lane_inst_per_px") is None
    if bench.profiled("fused_extract_16384_u16", "lane_inst_per_px") is not None:
        assert bench.profiled("fused_extract_16384_u16", "no_such_field") is None


def test_peaks_reads_measured_file_or_falls_back():
    hbm, source, raw = bench.peaks()
    assert hbm > 1000
    assert source in ("measured", "fallback")
    if source == "measured":
        assert float(raw["hbm_gbs"]) == hbm
