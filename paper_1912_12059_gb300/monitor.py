"""Per-N-step diagnostics of a run as JSON lines (one JSON object per line).

`run_logged` advances a `nsk.Solver` (or anything with its `step`, `compute_dt`, `diagnostics`,
`E` and `npe`) in chunks of `every` LSRK4 steps and, after each chunk, writes one line with the
step count, the simulated time, the step size, the paper's diagnostics (mass, the total energy of
relaxation model II, ||rho - c|| in L2: Sec. 4, the energy functional of Eq.
pararelax_elliptical_energy_dynamic) and the chunk's wall time and DOF-updates/s. The arithmetic
of the diagnostics is the library's (nsk_diagnostics); this module only calls and formats.
"""
from __future__ import annotations

import json
import time


def run_logged(solver, nsteps, every, out, dt=None, cfl=None, t0=0.0, step0=0, sync=None):
    """Advance `nsteps` steps, logging every `every` steps to `out` (a path or a writable text
    file). Step size: the fixed `dt`, or with `cfl` the device's CFL step recomputed before every
    step (then the logged dt is the last chunk's mean). `sync` (optional) is called before each
    clock reading, e.g. torch.cuda.synchronize (the solver's calls already synchronise).
    Returns the list of logged records."""
    if (dt is None) == (cfl is None):
        raise ValueError("give exactly one of dt and cfl")
    if every < 1 or nsteps < 0:
        raise ValueError("every must be >= 1 and nsteps >= 0")
    own = isinstance(out, (str, bytes)) or hasattr(out, "__fspath__")
    fh = open(out, "w") if own else out
    records = []
    try:
        t, step = float(t0), int(step0)
        nodes = solver.E * solver.npe
        done = 0
        while done < nsteps:
            n = min(every, nsteps - done)
            if sync:
                sync()
            c0 = time.perf_counter()
            if dt is not None:
                solver.step(dt, n)
                h = dt
                t += n * dt
            else:
                h_sum = 0.0
                for _ in range(n):
                    h_i = solver.compute_dt(cfl)
                    solver.step(h_i, 1)
                    h_sum += h_i
                h = h_sum / n
                t += h_sum
            if sync:
                sync()
            wall = time.perf_counter() - c0
            done += n
            step += n
            mass, energy, l2 = solver.diagnostics()
            rec = {"step": step, "t": t, "dt": h, "mass": mass, "energy": energy, "l2_rho_minus_c": l2,
                   "wall_s": wall, "dof_updates_per_s": nodes * 5 * n / wall if wall > 0 else None}
            fh.write(json.dumps(rec) + "\n")
            fh.flush()
            records.append(rec)
    finally:
        if own:
            fh.close()
    return records
