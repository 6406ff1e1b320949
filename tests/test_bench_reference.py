"""The reference arm of bench.py (--impl reference: the FP64 CPU oracle, OpenMP build on the
host cores) on the CPU: one JSON line with the keys of the benchmark contract, on rank 0 only;
every step one timed LSRK4 step of the oracle, on the workload's own mesh or, above the size
bound, on a labelled sample of it. Small meshes keep the test short; the arithmetic is the same."""
import dataclasses
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def _small(ne):
    wl = bench.workload_by_name("collision3d")
    return dataclasses.replace(wl, nelem=(ne,) * 3, name=f"{wl.name}_resized_E{ne}")


def _run(wl, capsys, steps=2, warmup=1):
    rc = bench.run_reference(bench.argparse.Namespace(gpus=1, steps=steps, warmup=warmup), wl, 0, 1)
    out = capsys.readouterr().out.strip().splitlines()
    assert rc == 0 and len(out) == 1
    return json.loads(out[0])


def test_reference_arm_prints_the_contract_line(capsys):
    wl = _small(8)
    line = _run(wl, capsys)
    assert line["impl"] == "reference" and line["metric"] == "DOF-updates/s" and line["unit"] == "DOF-updates/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 2 and line["warmup"] == 1 and line["dtype"] == "f64" and line["vs_baseline"] is None
    # the workload's own mesh: value and ms_per_step describe the same measured steps
    assert line["sample"]["full_workload"] is True and line["sample"]["nodes"] == wl.dofs
    assert abs(line["ms_per_step"] - wl.dofs * 5 / line["value"] * 1e3) < 1e-9 * line["ms_per_step"]
    assert line["config"]["workload"] == wl.name and line["config"]["dofs_per_gpu"] == wl.dofs
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_labels_its_sample(monkeypatch, capsys):
    monkeypatch.setattr(bench, "REFERENCE_FULL_MAX_NODES", 30000)
    monkeypatch.setattr(bench, "REFERENCE_SAMPLE_NELEM", {3: (8, 8, 8)})
    wl = _small(12)
    line = _run(wl, capsys, steps=1, warmup=0)
    assert line["sample"] == {"nelem": [8, 8, 8], "nodes": 512 * 64, "full_workload": False}
    assert abs(line["ms_per_step"] - 512 * 64 * 5 / line["value"] * 1e3) < 1e-9 * line["ms_per_step"]
    assert line["config"]["workload"] == wl.name and "8x8x8-element" in line["cpu_baseline"]["sample"]


def test_reference_arm_is_silent_on_other_ranks(capsys):
    wl = bench.workload_by_name("collision3d")
    assert bench.run_reference(bench.argparse.Namespace(gpus=2, steps=1, warmup=0), wl, 1, 2) == 0
    assert capsys.readouterr().out == ""
