"""bench.py's command line on the CPU: every workload and option combination the benchmark
offers parses, and main() runs the reference arm end to end (the oracle sample shortened for
the test)."""
import json
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

COMMANDS = [
    [],
    ["--gpus", "1", "--steps", "20", "--warmup", "5"],
    ["--impl", "reference", "--steps", "2", "--warmup", "3"],
    ["--steps", "2", "--warmup", "3", "--no-variants", "--no-cpu-baseline", "--nelem", "40", "--schedule", "256,0"],
    ["--precision", "fp32", "--steps", "2", "--warmup", "3", "--no-variants", "--nelem", "40",
     "--schedule", "256,0"],
    ["--workload", "batch", "--steps", "10", "--warmup", "3"],
    ["--workload", "closure", "--nelem", "48", "--train-steps", "500", "--samples", "20000"],
    ["--workload", "gemm", "--rows", "60000", "--steps", "5", "--warmup", "3"],
    ["--workload", "fp32err", "--steps", "5000"],
    ["--workload", "esdirk"],
    ["--workload", "riemann1d"],
    ["--workload", "coalescence2d", "--steps", "20"],
    ["--workload", "interface1d", "--steps", "2000"],
    ["--workload", "fp64peak"],
]


@pytest.mark.parametrize("args", COMMANDS, ids=[" ".join(a) or "default" for a in COMMANDS])
def test_command_parses(args):
    bench.make_parser().parse_args(args)


def test_main_runs_the_reference_arm(monkeypatch, capsys):
    monkeypatch.setattr(bench, "REFERENCE_FULL_MAX_NODES", 30000)
    monkeypatch.setattr(bench, "REFERENCE_SAMPLE_NELEM", {3: (8, 8, 8)})
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["warmup"] == 3 and line["steps"] == 1  # W >= 3 enforced
    assert line["config"]["workload"] == bench.workload_by_name("collision3d").name
