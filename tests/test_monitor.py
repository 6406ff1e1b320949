"""The JSON-lines run logger on the CPU, with a stand-in for the solver that records its calls
(the solver's own arithmetic is tested on the GPU)."""
import io
import json

import pytest

from paper_1912_12059_gb300 import monitor


class FakeSolver:
    E, npe = 10, 8

    def __init__(self):
        self.calls = []
        self.steps = 0

    def step(self, dt, n):
        self.calls.append(("step", dt, n))
        self.steps += n

    def compute_dt(self, cfl):
        self.calls.append(("dt", cfl))
        return 1e-3 * cfl

    def diagnostics(self):
        return 1.0 + self.steps, -2.0, 0.5


def test_fixed_dt_chunks_and_records(tmp_path):
    s = FakeSolver()
    path = tmp_path / "run.jsonl"
    recs = monitor.run_logged(s, 25, 10, path, dt=2e-4, t0=1.0, step0=5)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert lines == recs and [r["step"] for r in lines] == [15, 25, 30]
    assert [c[2] for c in s.calls] == [10, 10, 5]
    assert lines[-1]["t"] == pytest.approx(1.0 + 25 * 2e-4) and lines[0]["mass"] == 11.0
    assert set(lines[0]) == {"step", "t", "dt", "mass", "energy", "l2_rho_minus_c", "wall_s", "dof_updates_per_s"}


def test_cfl_steps_and_file_object():
    s = FakeSolver()
    buf = io.StringIO()
    recs = monitor.run_logged(s, 4, 2, buf, cfl=0.5)
    assert [c[0] for c in s.calls] == ["dt", "step"] * 4
    assert recs[0]["dt"] == pytest.approx(5e-4) and recs[-1]["t"] == pytest.approx(4 * 5e-4)
    assert len(buf.getvalue().splitlines()) == 2


def test_argument_checks():
    with pytest.raises(ValueError):
        monitor.run_logged(FakeSolver(), 1, 1, io.StringIO())
    with pytest.raises(ValueError):
        monitor.run_logged(FakeSolver(), 1, 0, io.StringIO(), dt=1e-3)
