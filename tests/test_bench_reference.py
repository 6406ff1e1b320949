"""The reference arm of bench.py (--impl reference: the FP64 CPU oracle timed on the host) on
the CPU: one JSON line with the keys of the benchmark contract, on rank 0 only. The oracle
sample is shortened for the test; the arithmetic is the same."""
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample", lambda wl, target_s=15.0: real(wl, target_s=0.05))
    wl = bench.workload_by_name("collision3d")
    rc = bench.run_reference(bench.argparse.Namespace(gpus=1, steps=2, warmup=1), wl, 0, 1)
    out = capsys.readouterr().out.strip().splitlines()
    assert rc == 0 and len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == "DOF-updates/s" and line["unit"] == "DOF-updates/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 2 and line["warmup"] == 1 and line["dtype"] == "f64" and line["vs_baseline"] is None
    assert abs(line["ms_per_step"] - wl.dofs * 5 / line["value"] * 1e3) < 1e-9 * line["ms_per_step"]
    assert line["config"]["workload"] == wl.name
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks(capsys):
    wl = bench.workload_by_name("collision3d")
    assert bench.run_reference(bench.argparse.Namespace(gpus=2, steps=1, warmup=0), wl, 1, 2) == 0
    assert capsys.readouterr().out == ""
