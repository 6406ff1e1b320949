"""bench.py's command line on the CPU: every `python bench.py ...` command recorded in the
profile summaries and the documentation parses, and main() runs the reference arm end to end
(the oracle sample shortened for the test)."""
import json
import re
import shlex
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402


def _recorded_commands():
    cmds = []
    for doc in sorted((ROOT / "profiles").glob("*.md")) + [ROOT / "DESIGN.md", ROOT / "README.md"]:
        text = doc.read_text().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^`\n>|&;)'#]*)", text):
            args = shlex.split(m.group(1).strip().rstrip("."))
            cmds.append((doc.name, args))
    return cmds


COMMANDS = _recorded_commands()


def test_commands_were_found():
    assert len(COMMANDS) >= 8


@pytest.mark.parametrize("doc,args", COMMANDS, ids=[f"{d}:{' '.join(a)}" for d, a in COMMANDS])
def test_recorded_command_parses(doc, args):
    bench.make_parser().parse_args(args)


def test_main_runs_the_reference_arm(monkeypatch, capsys):
    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample", lambda wl, target_s=15.0: real(wl, target_s=0.05))
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["warmup"] == 3 and line["steps"] == 1  # W >= 3 enforced
    assert line["config"]["workload"] == bench.workload_by_name("collision3d").name
