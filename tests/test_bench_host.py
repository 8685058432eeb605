"""bench.py host-side contract on CPU: the reference arm (the oracle, timed on host cores) prints
one JSON line with the contract's keys, and the replica value is the whole-job rate."""
import io
import json
import os
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_contract_line(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = SimpleNamespace(volumes=1, ref_sample=20000, warmup=1, steps=1, gpus=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gpoints/s" and d["value"] > 0
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
              "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_replica_value_is_whole_job_rate():
    import bench
    # N ranks each processing n points, slowest rank 20 ms -> N * n / 0.020 points/s
    assert abs(bench.replica_value(4, 1_000_000, 20.0) - 4 * 1e6 / 0.020 / 1e9) < 1e-12
