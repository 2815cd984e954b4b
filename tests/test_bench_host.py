"""bench.py's host-side contract, without a GPU: the reference arm (the oracle
timed as it stands on the host cores) prints one JSON line with the keys the
bench line carries, and the traffic record is only used when it was taken on
the current pass-kernel sources."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "7",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference"
    assert rec["steps"] == 2 and rec["warmup"] == 1 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"]["value"] == rec["value"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0


def test_traffic_record_is_keyed_on_the_pass_sources():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    with open(os.path.join(ROOT, "profiles", "pass_kernel_traffic.json")) as f:
        rec = json.load(f)
    digest = bench.pass_source_digest()
    for dtype, ent in rec.items():
        got = bench.traffic_record(dtype)
        if ent.get("source_sha256_16") == digest:
            assert got is not None and got["bytes_per_launch"] == ent["bytes_per_launch"]
        else:
            assert got is None
    assert bench.traffic_record("no-such-dtype") is None
