"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract; it needs no GPU, so it runs here on a small workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_line_keeps_the_contract():
    lines = _run({}, "--rays", "64", "--slices", "8", "--steps", "2", "--warmup", "1")
    assert len(lines) == 1
    d = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("volume-64 (8 slices x 64 angles x 64 rays")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_ranks_other_than_zero_do_no_work():
    assert _run({"WORLD_SIZE": "2", "RANK": "1"}, "--rays", "64", "--steps", "1", "--warmup", "1") == []


def test_stored_traffic_applies_only_to_its_device_code_and_shape(monkeypatch):
    """The ncu traffic record is used only while the kernels' device code hashes
    to the record's value and the benchmark runs the captured launch shape;
    any other shape field (layout, chunk, block order, radix, gather form),
    geometry or device code gives no traffic figure."""
    sys.path.insert(0, ROOT)
    import bench
    rec = bench.CAPTURED_TRAFFIC[0]
    monkeypatch.setattr(bench, "device_code_sha", lambda: rec["sha"])
    shape = dict(rec["shape"], max_lanes=2)
    assert bench.captured_traffic("k_grid_col", rec["rays"], rec["pad"], shape) == rec["bytes"]["k_grid_col"]
    for k, other in (("layout", "packed"), ("chunk_pairs", 4), ("pair_fast", 0), ("max_radix", 8), ("grid_xchg", 0)):
        if shape[k] != other:
            assert bench.captured_traffic("k_grid_col", rec["rays"], rec["pad"], dict(shape, **{k: other})) is None, k
    assert bench.captured_traffic("k_grid_col", rec["rays"] // 2, rec["pad"], shape) is None
    monkeypatch.setattr(bench, "device_code_sha", lambda: "0" * 64)
    assert bench.captured_traffic("k_grid_col", rec["rays"], rec["pad"], shape) is None
