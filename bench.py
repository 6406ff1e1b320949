#!/usr/bin/env python3
"""Benchmark of the explicit DGSEM hot path of the parabolic relaxation model
(arXiv:1912.12059, relaxation model II) on GB300.

A "step" is one five-stage LSRK4 step over the whole mesh (every stage: trace
prolongation, BR1 lifting, face fluxes, volume integral + surface lifting +
sources + RK update). The metric is DOF-updates/s = nodes x 5 stages x steps /
seconds, timed with CUDA events on the solver's stream with the state resident
in HBM. `e2e` repeats the measurement through the C ABI with the state in
pinned host memory, copied in before and read back after every step.

Default workload: 3D head-on droplet collision, 64^3 elements, N = 3 (16.8M
nodes x 5 variables), FP64, We = 40. Under torchrun each rank advances its own
instance (independent problems: weak scaling, no data-path collective).

`--impl reference` times the FP64 CPU oracle instead (test infrastructure of
this repository) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

MEASURED_PEAKS = ROOT / "MEASURED_PEAKS.json"
# FP64 and FP32 FMAs per SM and clock. GB300's nominal FP64 rate, 1.25 TFLOP/s, over 152 SMs x
# 2 flops x 2.07 GHz is 1.99: 2 DFMA per SM and clock; FP32: 128 FFMA per SM and clock. The
# nsk_measure_fma_rate probe measures both in every run (reported beside the derived peaks).
DFMA_PER_SM_CLK = 2
FFMA_PER_SM_CLK = 128
# Algorithmic (compulsory) bytes per node and stage: U and K read and written once, nvar values
# of 8 (FP64) or 4 (FP32) bytes each.
def compulsory_bytes(d, fp_bytes):
    return 4 * (d + 2) * fp_bytes


# DRAM bytes (read + write) per launch of a kernel at 64^3 elements, N = 3, from one ncu capture
# at 40^3 elements of the same kernel source, scaled by the element count; None once the kernel
# changed after the capture (then no traffic is claimed). FP64: k_volume (separate face pass,
# 11,671 + 9,600 B per element); FP32: the line schedule's volume kernel, k_volume_line
# (5.83 + 3.63 KB per element).
MEASURED_TRAFFIC = {("k_volume", 8, 262144): 5.576e9, ("k_volume", 4, 262144): 2.480e9}
TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at 40^3 elements, scaled to 64^3"


def alu_peak_tflops(sms, sm_mhz, fp64=True):
    """Peak FMA throughput: SMs x FMAs per SM and clock x 2 flops x SM clock (MHz)."""
    return sms * (DFMA_PER_SM_CLK if fp64 else FFMA_PER_SM_CLK) * 2 * sm_mhz * 1e6 / 1e12


def host_info():
    """Cores and CPU model of the host the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def workload_by_name(name):
    from paper_1912_12059_gb300 import inputs

    if name == "collision3d":
        return inputs.head_on_collision_3d(we=40.0)
    if name == "coalescence2d":
        return inputs.coalescence_2d(alpha=1e2)
    if name == "interface1d":  # Gauss-Legendre nodes: on Gauss-Lobatto nodes the run goes non-physical near t = 2e-3
        import dataclasses

        wl = inputs.static_interface_1d(node_type=0)
        return dataclasses.replace(wl, name=wl.name + "_GL")
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------- algorithmic cost model
def kernel_cost(kernel, d, n, fp_bytes, traces=0.0, sched=0):
    """Algorithmic (flops, bytes) per element of one stage kernel, counted from the kernel
    source: FMA = 2 flops, add/mul/div/sqrt = 1 (negations, compares and min/max are free);
    bytes = compulsory loads + stores. `traces`: fraction of the k_volume launches that also
    wrote the face traces of their output state (the next stage's prolongation: its flops and
    trace stores). FP64 traces carry 1/rho and 1/(3 - rho) (one division per trace node);
    FP32 kernels divide where FP64 reads those planes. sched = 2: the lean stage's kernels
    (k_lift: the lifting from the element's state, its own traces prolonged on chip, and the
    neighbours' state traces, storing only the viscous-flux traces; k_volume: that lifting again,
    the element's 2d face fluxes and the volume kernel, reading the state, the RK register and
    the neighbours' state and viscous-flux traces)."""
    npe, nfn, nv, nw, nf = n**d, n ** (d - 1), d + 2, d + 1, 2 * d
    if kernel == "k_block":  # one stage of the single-block kernel: its arrays stay on chip
        fl = sum(kernel_cost(k, d, n, fp_bytes, traces=traces)[0] for k in ("k_lift", "k_face", "k_volume"))
        return fl, 0.0
    if sched == 2 and kernel in ("k_lift", "k_volume"):
        xp = 2 if fp_bytes == 8 else 0
        prolong_own = kernel_cost("k_prolong", d, n, fp_bytes)[0]       # own traces on chip
        fl_lift = kernel_cost("k_lift", d, n, fp_bytes)[0] + prolong_own
        nbr = nf * nfn * (nv + xp)                                         # the neighbours' state traces
        if kernel == "k_lift":
            return fl_lift, fp_bytes * (nv * npe + nbr + nf * nfn * nw)
        fl_face = 2 * kernel_cost("k_face", d, n, fp_bytes)[0]            # each face by both elements
        fl_vol, _ = kernel_cost("k_volume", d, n, fp_bytes, traces=traces)  # its stress is the lifting's
        by = fp_bytes * (4 * nv * npe + nbr + nf * nfn * nw + traces * nf * nfn * (nv + xp))
        return fl_lift + fl_face + fl_vol, by
    fp64 = fp_bytes == 8
    trace_extra = 5 if fp64 else 0            # 3 - rho, rho (3 - rho), 1/x, two products
    stress = (d - 1) + d * (d - 1) // 2 + 3 * d  # div v, off-diagonal sums, diagonal sum + fma
    xp = 2 if fp64 else 0                     # FP64 trace planes 1/rho, 1/(3 - rho)
    if kernel == "k_prolong":
        return nf * nfn * (nv * 2 * n + trace_extra), fp_bytes * (nv * npe + nf * nfn * (nv + xp))
    nvf = d * (d + 1) // 2 + d                # viscous form: stress / mu and grad c
    if kernel == "k_lift":
        per_node = (d + 1) + d * nw * (2 * n + 4) + stress          # w = (m / rho, c); grad w; tau
        per_face = (3 * d + 1) + (0 if fp64 else 2)                  # 2 w* (and two reciprocals)
        fl = npe * per_node + nf * nfn * per_face + nf * nfn * nw * 2 * n
        by = fp_bytes * (nv * npe + 2 * nf * nfn * (nv + xp // 2) + nvf * npe + nf * nfn * nw)  # + 1/rho
        return fl, by
    if kernel == "k_face":
        eos = 18 if fp64 else 30                                     # both sides (FP32: + 1/rho)
        per_fn = eos + 6 + 1 + 7 + 5 * (d - 1) + 1 + 3 * (nv - 1)    # lambda (its v_k reused), 2 F* (LF), jump
        return d * nfn * per_fn, fp_bytes * d * nfn * (2 * (nv + xp) + 2 * nw + nv)
    if kernel == "k_volume":
        eos = 10 if fp64 else 8
        flux = d + 2 * d + d * (d - 1) // 2 + 2 * d * d              # v_a, F^c (each pair k < a once), F^c - mu tau
        per_node = eos + flux + nv * d * (2 * n + 4) + 2 + (2 * d + 4) + 4 * nv  # stress read, not formed
        by = fp_bytes * (nv * npe + nvf * npe + 2 * d * nfn * nv + 2 * nv * npe + nv * npe)
        return (npe * per_node + traces * nf * nfn * (nv * 2 * n + trace_extra),
                by + traces * fp_bytes * nf * nfn * (nv + xp))
    raise KeyError(kernel)


BATCH_KINDS = {0: "one launch per phase", 1: "persistent cooperative", 2: "instance launches"}


def pick_schedule(s, fixed):
    """The autotuner's stage schedule, or a fixed "TPB,FUSED" one (profiling runs: under a
    profiler the autotuner's timings are serialised and would pick another schedule); FUSED is
    0 (separate face pass), 1 (face fluxes in the volume kernel), 2 (the lean stage), 3 (the
    single-block schedule) or 4 (the line-per-thread FP32 kernels)."""
    if fixed:
        tpb, fused = (int(v) for v in fixed.split(","))
        s.set_schedule(tpb, fused)
        return tpb, fused
    tpb, fused, _ = s.autotune()
    return tpb, fused


def trace_fraction(prof):
    """Share of the k_volume launches that wrote the next stage's traces: every nsk_step call
    prolongs once at its start and skips the trace store in its last stage."""
    nv = prof.get("k_volume", (0.0, 0))[1]
    return (nv - prof.get("k_prolong", (0.0, 0))[1]) / nv if nv else 0.0


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = Path(tempfile.mkstemp(prefix="nsk_clocks_", suffix=".csv")[1])

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        rows = []
        try:
            for line in self.path.read_text().splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                self.path.unlink()
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle baseline
def oracle_sample(wl, target_s=15.0, parallel=False, ne=None):
    """Time the FP64 CPU oracle as it stands (plain build on one thread, or parallel=True: the
    OpenMP build of the same source on all host cores) on a bounded sample of the workload: the
    same N, parameters and initial-condition recipe on a smaller periodic mesh (the oracle's cost
    per node does not depend on the mesh spacing). Returns (DOF-updates/s, description, threads)."""
    import oracle as O

    ne = ne or {3: (8, 8, 8), 2: (32, 32), 1: (64,)}[wl.dim]
    o = O.Oracle(wl.dim, ne, [0.0] * wl.dim, [1.0] * wl.dim, wl.N, wl.node_type, T=wl.T, kappa=wl.kappa,
                 alpha=wl.alpha, beta=wl.beta, mu=wl.mu, parallel=parallel)
    U = wl.initial_state(o.coords())
    dt = o.timestep(U, wl.cfl)
    t0 = time.perf_counter()
    steps = 0
    while True:
        U = o.step(U, dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el > target_s or steps >= 1000:
            break
    nodes = o.E * o.npe
    rate = nodes * 5 * steps / el
    threads = O.threads(parallel)
    return rate, f"{steps} LSRK4 steps of the oracle ({'OpenMP build, ' if parallel else 'plain build, '}" \
                 f"{threads} thread{'s' if threads > 1 else ''}) on a {'x'.join(map(str, ne))}-element periodic " \
                 f"box (N={wl.N}, {nodes} nodes, same parameters and initial-condition recipe), {el:.1f} s", threads


def cpu_baselines(wl, seconds):
    """The oracle on the host: all cores (OpenMP build) and one core (plain build), with the host's
    core count and CPU model."""
    rate_p, desc_p, thr = oracle_sample(wl, target_s=seconds, parallel=True,
                                        ne={3: (16, 16, 16), 2: (64, 64), 1: (64,)}[wl.dim])
    rate_1, desc_1, _ = oracle_sample(wl, target_s=seconds)
    return {"value": rate_p, "unit": "DOF-updates/s", "cores": thr, "kind": "oracle", "sample": desc_p,
            "host": host_info(),
            "single_core": {"value": rate_1, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
                            "sample": desc_1}}


# the reference arm runs the workload's own mesh up to this many nodes, else this sample of it
REFERENCE_FULL_MAX_NODES = 1 << 22
REFERENCE_SAMPLE_NELEM = {3: (32, 32, 32), 2: (128, 128), 1: (64,)}


def run_reference(args, wl, rank, world):
    """--impl reference: the FP64 CPU oracle (OpenMP build of the plain source, all host cores),
    rank 0 only. Every step is one LSRK4 step of the oracle on the workload's own mesh when it
    holds at most 2^22 nodes, else on a bounded sample of it (the same N, parameters and
    initial-condition recipe on the periodic box REFERENCE_SAMPLE_NELEM); each step is
    timed, ms_per_step is the measured mean and value the sample's DOF-updates/s."""
    if rank != 0:
        return 0
    import oracle as O

    full = wl.dofs <= REFERENCE_FULL_MAX_NODES
    ne = tuple(wl.nelem) if full else REFERENCE_SAMPLE_NELEM[wl.dim]
    o = O.Oracle(wl.dim, ne, [0.0] * wl.dim, [1.0] * wl.dim, wl.N, wl.node_type, T=wl.T, kappa=wl.kappa,
                 alpha=wl.alpha, beta=wl.beta, mu=wl.mu, parallel=True)
    U = wl.initial_state(o.coords())
    dt = o.timestep(U, wl.cfl)
    for _ in range(args.warmup):
        U = o.step(U, dt, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        U = o.step(U, dt, 1)
        times.append(time.perf_counter() - t0)
    nodes = o.E * o.npe
    ms_per_step = 1e3 * sum(times) / max(len(times), 1)
    value = nodes * 5 / (ms_per_step / 1e3)
    threads = O.threads(True)
    sample = (f"every step one LSRK4 step of the oracle (OpenMP build, {threads} threads) on "
              + ("the workload's own mesh" if full else
                 f"a {'x'.join(map(str, ne))}-element periodic box of the workload (same N = {wl.N}, parameters "
                 f"and initial-condition recipe; {nodes} of the workload's {wl.dofs} nodes)"))
    line = {
        "impl": "reference", "metric": "DOF-updates/s", "value": value, "unit": "DOF-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "dofs_per_gpu": wl.dofs, "N": wl.N, "nelem": list(wl.nelem)},
        "sample": {"nelem": list(ne), "nodes": nodes, "full_workload": full},
        "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def aggregate_ranks(ms, e2e_s, nodes, world, device):
    """Whole-job figures of a weak-scaling run (every rank advances its own instance): the
    slowest rank's device time and end-to-end time, and the nodes of all ranks (collectives over
    the default process group, on tensors of `device`)."""
    if world <= 1:
        return ms, e2e_s, nodes
    import torch
    import torch.distributed as dist

    tt = torch.tensor([ms, e2e_s], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    nn = torch.tensor([float(nodes)], device=device, dtype=torch.float64)
    dist.all_reduce(nn, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(nn[0])


def run_gpu(args, wl, rank, world):
    import torch
    import torch.distributed as dist

    from paper_1912_12059_gb300 import nsk
    from paper_1912_12059_gb300.build import build_library

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not (ROOT / "paper_1912_12059_gb300" / "libnsk.so").exists():
        build_library()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.Stream()
    prec = nsk.NSK_FP32_MIXED if args.precision == "fp32" else nsk.NSK_FP64
    s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type, prec,
                   stream=stream.cuda_stream)
    s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    x = s.node_coords()
    U0 = wl.initial_state(x)
    s.set_state(U0)
    tpb, fused = pick_schedule(s, args.schedule)  # setup: the fastest stage schedule for this mesh
    dt = s.compute_dt(wl.cfl)
    nodes = s.E * s.npe
    # FMA throughput of this GPU, measured with its clocks sampled (cross-check of the derived
    # FP64 peak of the roofline)
    with ClockSampler(local) as pclk:
        probe64, _ = nsk.measure_fma_rate(nsk.NSK_FP64, iters=1 << 17)
        probe64 = max(probe64, nsk.measure_fma_rate(nsk.NSK_FP64, iters=1 << 17)[0])
    probe_clk = pclk.summary()["sm_mhz"]

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    s.step(dt, args.warmup)
    # timed region: device-resident state
    s.set_profiling(True)
    s.get_profile(reset=True)
    launches0 = s.launch_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        s.step(dt, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = s.launch_count - launches0
    prof = s.get_profile(reset=True)
    s.set_profiling(False)
    clocks = clk.summary()
    U_after = s.get_state() if (prec == nsk.NSK_FP64 and not args.no_variants and world == 1) else None

    # end to end through the C ABI: pinned host state in, step, state out, every step
    U_host = torch.from_numpy(s.get_state()).pin_memory()
    nbytes = U_host.numel() * 8
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):  # nsk_step_host: the state in, one step, the state out
        s.step_host(U_host, dt, 1)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()

    # aggregate over ranks: total units / max time
    t_max, e2e_max, total_nodes = aggregate_ranks(ms, e2e_s, nodes, world, "cuda")
    value = total_nodes * 5 * args.steps / (t_max / 1e3)
    e2e_value = total_nodes * 5 * e2e_steps / e2e_max

    # roofline of the dominant kernel
    fp_bytes = 8 if prec == nsk.NSK_FP64 else 4
    name, (kms, kcnt) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = kms / max(kcnt, 1)
    flops_e, bytes_e = kernel_cost(name, wl.dim, wl.N + 1, fp_bytes, traces=trace_fraction(prof), sched=fused)
    if name == "k_block":  # the single-block kernel runs every stage of the timed call in one launch
        flops_e *= 5 * args.steps
    peaks = json.loads(MEASURED_PEAKS.read_text()) if MEASURED_PEAKS.exists() else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured (STREAM-style copy)" if "hbm_gbs" in peaks else "fallback"
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = clocks["sm_max_mhz"] or float(peaks.get("sm_max_mhz", 2070.0))
    traffic = MEASURED_TRAFFIC.get((name, fp_bytes, s.E))
    if prec == nsk.NSK_FP64:
        peak = alu_peak_tflops(sms, max_mhz, fp64=True)
        achieved = flops_e * s.E / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": name,
                "peak_source": f"derived: {sms} SMs x {DFMA_PER_SM_CLK} DFMA/clk x 2 flop x {max_mhz:.0f} MHz "
                               "(max SM clock); the probe measured in this run is probe_fp64_tflops",
                "probe_fp64_tflops": probe64, "probe_sm_mhz_median": probe_clk,
                "algorithmic_per_launch": flops_e * s.E, "unit_count": "counted flops of the kernel source per element"}
    else:
        achieved = bytes_e * s.E / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": name, "peak_source": hbm_src,
                "algorithmic_per_launch": bytes_e * s.E}
    roof["traffic_source"] = TRAFFIC_SOURCE if traffic is not None else None
    # the whole step against HBM on the compulsory bytes (U and K read and written once per stage)
    step_bytes = compulsory_bytes(wl.dim, fp_bytes) * total_nodes * 5 * args.steps
    roof_step = {"bound": "hbm", "bytes_per_node_stage": compulsory_bytes(wl.dim, fp_bytes),
                 "achieved": step_bytes / (t_max / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                 "frac": step_bytes / (t_max / 1e3) / 1e9 / hbm, "peak_source": hbm_src}
    kernels = {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-30)} for k, v in prof.items()}
    s.close()
    variants = {}
    if U_after is not None:
        variants["fp32_mixed"] = measure_fp32_variant(args, wl, stream, U0, U_after, dt, peaks)
        variants["fp64_hllc"] = measure_hllc_variant(args, wl, stream, U0, U_after, dt)
        variants["fp64_original_nsk"] = measure_nsk_variant(args, wl, stream, U0, dt)
        variants["interface1d"] = measure_interface1d_variant(args, stream)
        variants["coalescence2d"] = measure_coalescence2d_variant(args, stream, peaks)
        variants["batch32"] = measure_batch_variant(args)
        variants["closure96"] = measure_closure_variant(args)
        variants["riemann1d_subcell"] = measure_subcell_variant(args, stream)
        variants["esdirk4_implicit"] = measure_esdirk_variant(args, stream)

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(wl, args.cpu_seconds)
    line = {
        "metric": "DOF-updates/s", "value": value, "unit": "DOF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == nsk.NSK_FP64 else "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "dofs_per_gpu": nodes, "N": wl.N, "nelem": list(wl.nelem),
                   "precision": args.precision, "dt": dt, "schedule": {"tpb": tpb, "fused_face": fused},
                   "l2": "state larger than L2 (inputs > 129 MB)"
                   if nodes * (wl.dim + 2) * fp_bytes > 129e6 else "state fits L2"},
        "e2e": {"value": e2e_value, "unit": "DOF-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_step_hbm": roof_step,
        "kernels": kernels,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "cpu_baseline": cpu,
        "variants": variants,
    }
    print(json.dumps(line))
    return 0


def run_batch(args, rank, world):
    """32 uneven 3D collision instances (16^3..48^3 elements, N in {3,4}) advanced together
    (CUDA-graph replay of the five stage launches under the autotuned batch schedule)."""
    import torch

    from paper_1912_12059_gb300 import nsk
    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        v = measure_batch_variant(args, n=args.batch)
    clocks = clk.summary()
    small = batch_vs_sequential_small(nsk, nsk.NSK_FP32_MIXED)
    if rank != 0:
        return 0
    line = {
        "metric": "DOF-updates/s", "value": v["value"], "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(v, small_instances=small, l2="state larger than L2"),
        "gpu_launches": v["gpu_launches"],
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "e2e": None, "roofline": None, "cpu_baseline": None,
    }
    print(json.dumps(line))
    return 0


def batch_vs_sequential_small(nsk, prec, n=64, steps=20):
    """Serving-style comparison: many small instances (6^3..12^3 elements), batched graph replay
    vs stepping the instances one after another."""
    import torch

    from paper_1912_12059_gb300 import inputs

    wls = inputs.serving_batch_3d(n, seed=inputs.SEED + 7, e_range=(6, 12))
    solvers = []
    for wl in wls:
        s = nsk.Solver(3, wl.nelem, wl.N, [0, 0, 0], [1, 1, 1], 0, prec)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        s.set_state(wl.initial_state(s.node_coords()))
        s.compute_dt(wl.cfl)
        solvers.append(s)
    nodes = sum(s.E * s.npe for s in solvers)
    b = nsk.Batch(solvers)
    tpb, fused, persistent, _ = b.autotune()
    b.step(3)
    ms = b.step(steps, timings=True)
    batched = nodes * 5 * steps / (sum(ms) / 1e3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for s in solvers:
            s.step(s.compute_dt(0.5), 1)
    torch.cuda.synchronize()
    seq = nodes * 5 * steps / (time.perf_counter() - t0)
    b.close()
    for s in solvers:
        s.close()
    sm = sorted(ms)
    return {"instances": n, "nodes_total": nodes, "batched_value": batched, "sequential_value": seq,
            "schedule": {"tpb": tpb, "fused_face": fused, "kind": BATCH_KINDS[persistent]},
            "step_latency_ms_p50": sm[len(sm) // 2], "step_latency_ms_p99": sm[-1]}


def measure_nsk_variant(args, wl, stream, U0, dt):
    """The original third-order NSK equations (state rho, m; second BR1 lifting for lap rho) on the
    same mesh and initial density and momentum, at the same dt: cost per step against model II,
    and the explicit step size each model's own bound allows there."""
    import torch

    from paper_1912_12059_gb300 import nsk

    s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type,
                   nsk.NSK_FP64, stream=stream.cuda_stream)
    s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    s.set_model(nsk.NSK_MODEL_NSK)
    s.set_state(np.ascontiguousarray(U0[:wl.dim + 1]))
    tpb, _ = pick_schedule(s, args.schedule)
    dt_own = s.compute_dt(wl.cfl)
    out = {"dtype": "f64", "model": "original NSK", "schedule": {"tpb": tpb}, "dt_model_ii": dt,
           "dt_own_bound": dt_own}
    try:
        s.step(dt, args.warmup)
        s.set_profiling(True)
        s.get_profile(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = s.get_profile(reset=True)
        out.update({"value": wl.dofs * 5 * args.steps / (ms / 1e3), "unit": "DOF-updates/s",
                    "ms_per_step": ms / args.steps,
                    "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1]} for k, v in prof.items()}})
    except nsk.NskError as ex:  # the central flux of the third-order system does not damp
        out["error"] = str(ex)
    s.close()
    return out


def measure_subcell_variant(args, stream):
    """The 1D multiphase Riemann problem of Sec. 4 in the sharp-interface limit with FV sub-cell
    shock capturing and Dirichlet boundaries (nsk_set_subcell, nsk_set_dirichlet): the paper's
    configuration (200 elements, N = 3, eps = 1e-3, HLLC, Persson thresholds -6 / -8) run to
    t = 0.11 at CFL 0.1 (time to solution; dt recomputed every 100 steps), and the same problem
    on 2^20 elements for throughput (fixed dt, CUDA events around the timed steps)."""
    import torch

    from paper_1912_12059_gb300 import inputs, nsk

    wl = inputs.riemann_1d_sharp(eps=1e-3)
    x = wl.extra

    def make(nelem):
        s = nsk.Solver(1, (nelem,), wl.N, [0.0], [1.0], wl.node_type, nsk.NSK_FP64, stream=stream.cuda_stream)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        s.set_flux(nsk.NSK_FLUX_HLLC)
        s.set_subcell(True, x["ind_upper"], x["ind_lower"])
        left, right = (x["rho_left"], 0.0, x["rho_left"]), (x["rho_right"], 0.0, x["rho_right"])
        s.set_dirichlet(left, right)
        s.set_state(inputs.riemann_1d(s.node_coords(), x["rho_left"], x["rho_right"], x["x0"]))
        return s

    out = {"workload": wl.name, "dtype": "f64", "flux": "hllc", "boundaries": "dirichlet",
           "indicator_thresholds": [x["ind_upper"], x["ind_lower"]]}
    s = make(wl.n_elem)
    t, steps, t_end = 0.0, 0, x["t_end"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    while t < t_end * (1 - 1e-12):
        dt = s.compute_dt(wl.cfl)
        n = min(100, int(math.ceil((t_end - t) / dt)))
        dt = min(dt, (t_end - t) / n)
        s.step(dt, n)
        t += n * dt
        steps += n
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    flags, _ = s.subcell()
    U = s.get_state()
    out["time_to_solution"] = {"t_end": t_end, "steps": steps, "wall_ms": ms, "ms_per_step": ms / steps,
                               "value": wl.dofs * 5 * steps / (ms / 1e3), "unit": "DOF-updates/s",
                               "subcell_elements_at_end": int(flags.sum()),
                               "rho_range_at_end": [float(U[0].min()), float(U[0].max())],
                               "launch": "one cooperative launch per nsk_step call"}
    # the same mesh with dt recomputed before every step: one launch per kernel and stage
    n = 200
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(-wl.cfl, n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["per_kernel_launches"] = {"steps": n, "ms_per_step": ms / n, "launches_per_step": 23,
                                  "value": wl.dofs * 5 * n / (ms / 1e3), "unit": "DOF-updates/s"}
    s.close()
    big = 1 << 20
    s = make(big)
    dt = s.compute_dt(wl.cfl)
    s.step(dt, args.warmup)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    flags, _ = s.subcell()
    nodes = big * (wl.N + 1)
    out["throughput"] = {"nelem": big, "nodes": nodes, "steps": args.steps, "ms_per_step": ms / args.steps,
                         "value": nodes * 5 * args.steps / (ms / 1e3), "unit": "DOF-updates/s",
                         "subcell_elements": int(flags.sum()), "launches_per_step": 21}
    s.close()
    return out


def measure_esdirk_variant(args, stream):
    """Implicit ESDIRK4 with Jacobian-free Newton-Krylov (nsk_step_esdirk) against the explicit
    LSRK4 over the same simulated time, on the 1D static phase interface (64 elements, N = 3,
    kappa = 1e-4), in two regimes of the c equation's stiffness alpha/beta:
      - mild, alpha = 100, beta = 1e-2, mu = 1e-2: T = 100 explicit CFL-0.5 steps, advanced by one
        implicit step of 100x and by ten of 10x the explicit step;
      - stiff, the paper's alpha = 1e3, beta = 1e-3, mu = 1e-3 (explicit dt bound by the source):
        T = 1000 explicit steps, advanced by one implicit step of 1000x and by ten of 100x;
    each without and with the element-block preconditioner: wall time, residual evaluations (those
    that build the blocks included), Newton and Krylov iterations, and the density L2 difference to
    the explicit run."""
    import torch

    from paper_1912_12059_gb300 import inputs, nsk

    E, N = 64, 3

    def compare(prm, n_explicit, factors):
        def make():
            s = nsk.Solver(1, (E,), N, [0.0], [1.0], 0, nsk.NSK_FP64, stream=stream.cuda_stream)
            s.set_params(**prm)
            s.set_state(inputs.slab_1d(s.node_coords(), inputs.PAPER_RHO_VAP, inputs.PAPER_RHO_LIQ, prm["kappa"]))
            return s

        s = make()
        dte = s.compute_dt(0.5)
        out = {"workload": f"static_interface_1d_E{E}_N{N}_alpha{prm['alpha']:g}_beta{prm['beta']:g}",
               "explicit_dt": dte, "simulated_time": n_explicit * dte, "newton_tol": 1e-10, "krylov_tol": 1e-3,
               "krylov_dim": 30}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.step(dte, 3)  # warm-up
        s.close()
        s = make()
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(dte, n_explicit)
        e1.record(stream)
        torch.cuda.synchronize()
        ref = s.get_state()
        out["explicit_lsrk4"] = {"steps": n_explicit, "wall_ms": e0.elapsed_time(e1),
                                 "rhs_evaluations": 5 * n_explicit}
        s.close()
        for pc in (False, True):
            for fac in factors:
                s = make()
                torch.cuda.synchronize()
                t0 = time.time()
                st = s.step_esdirk(fac * dte, n_explicit // fac, newton_tol=1e-10, krylov_tol=1e-3, krylov_dim=30,
                                   block_precond=pc)
                torch.cuda.synchronize()
                ms = (time.time() - t0) * 1e3
                U = s.get_state()
                err = float(np.sqrt(((U[0] - ref[0]) ** 2).sum() / (ref[0] ** 2).sum()))
                out[f"esdirk4_{fac}x" + ("_block_precond" if pc else "")] = {
                    "steps": n_explicit // fac, "wall_ms": ms, "rhs_evaluations": st["rhs"],
                    "newton": st["newton"], "krylov": st["krylov"], "failed": st["failed"],
                    "density_l2_rel_diff_vs_explicit": err}
                s.close()
        return out

    out = compare(dict(T=0.85, kappa=1e-4, alpha=100.0, beta=1e-2, mu=1e-2), 100, (100, 10))
    out["stiff_paper_parameters"] = compare(dict(T=0.85, kappa=1e-4, alpha=1e3, beta=1e-3, mu=1e-3), 1000,
                                            (1000, 100))
    return out


def measure_hllc_variant(args, wl, stream, U0, U_lf_after, dt):
    """The FP64 path with the HLLC face flux instead of local Lax-Friedrichs on the same workload:
    throughput, per-kernel times, and the density L2 difference to the Lax-Friedrichs run after
    the same steps (two consistent schemes: a measure of the flux's dissipation, not an error)."""
    import torch

    from paper_1912_12059_gb300 import nsk

    s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type,
                   nsk.NSK_FP64, stream=stream.cuda_stream)
    s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    s.set_flux(nsk.NSK_FLUX_HLLC)
    s.set_state(U0)
    tpb, fused = pick_schedule(s, args.schedule)
    s.step(dt, args.warmup)
    s.set_profiling(True)
    s.get_profile(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.get_profile(reset=True)
    U = s.get_state()
    s.close()
    diff = float(np.sqrt(((U[0] - U_lf_after[0]) ** 2).sum() / (U_lf_after[0] ** 2).sum()))
    return {"value": wl.dofs * 5 * args.steps / (ms / 1e3), "unit": "DOF-updates/s", "ms_per_step": ms / args.steps,
            "dtype": "f64", "flux": "hllc", "density_l2_rel_diff_vs_lf": diff,
            "schedule": {"tpb": tpb, "fused_face": fused},
            "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1]} for k, v in prof.items()}}


def _timed_steps(s, stream, dt, n):
    """Wall ms of n steps of a solver, CUDA events on its stream."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(dt, n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_interface1d_variant(args, stream):
    """The 1D static phase interface (64 elements, N = 3; kappa 1e-4, alpha 1e3, beta 1e-3,
    mu 1e-3) at CFL 0.5: on Gauss-Legendre nodes (the paper's) its full 2000 LSRK4 steps; on
    Gauss-Lobatto nodes, as the workload names them, 800 steps: the collocated Lobatto scheme
    goes non-physical near t = 2e-3 (about 900 steps) on this interface, in the oracle as on the
    GPU and at any step size. Wall time and rate, and the oracle's time for the same run on one
    host core (the CPU baseline of this workload)."""
    import dataclasses

    from paper_1912_12059_gb300 import inputs, nsk

    out = {}
    for nt, tag, steps in ((0, "gauss_legendre", 2000), (1, "gauss_lobatto", 800)):
        wl = dataclasses.replace(inputs.static_interface_1d(node_type=nt), steps=steps)
        s = nsk.Solver(1, wl.nelem, wl.N, [0.0], [1.0], nt, nsk.NSK_FP64, stream=stream.cuda_stream)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        U0 = wl.initial_state(s.node_coords())
        s.set_state(U0)
        tpb, fused = pick_schedule(s, "")  # the single-block schedule where it is fastest
        dt = s.compute_dt(wl.cfl)
        s.step(dt, 3)
        s.set_state(U0)
        n0 = s.launch_count
        ms = _timed_steps(s, stream, dt, wl.steps)
        launches = s.launch_count - n0
        m0 = s.diagnostics()[0]
        s.close()
        out[tag] = {"workload": wl.name + ("" if nt == 1 else "_GL"), "steps": wl.steps, "dt": dt, "wall_ms": ms,
                    "ms_per_step": ms / wl.steps, "value": wl.dofs * 5 * wl.steps / (ms / 1e3),
                    "unit": "DOF-updates/s", "dtype": "f64", "mass": m0,
                    "schedule": {"tpb": tpb, "fused_face": fused}, "gpu_launches": launches}
        if not args.no_cpu_baseline:
            import oracle as O

            o = O.Oracle(1, wl.nelem, [0.0], [1.0], wl.N, nt, T=wl.T, kappa=wl.kappa, alpha=wl.alpha,
                         beta=wl.beta, mu=wl.mu)
            t0 = time.perf_counter()
            o.step(U0, dt, wl.steps)
            el = time.perf_counter() - t0
            out[tag]["cpu_baseline"] = {"value": wl.dofs * 5 * wl.steps / el, "unit": "DOF-updates/s", "cores": 1,
                                        "kind": "oracle", "sample": f"the full {wl.steps}-step run, {el:.2f} s"}
    return out


def measure_coalescence2d_variant(args, stream, peaks):
    """2D coalescence of two droplets (128^2 elements, N = 4, radii 0.15 / 0.12, +-1e-4 noise) at
    alpha = 1e2, 1e3, 1e4: FP64 rate over 200 steps at the CFL-0.5 step of each, against HBM on
    the compulsory 128 B per node and stage; the oracle (OpenMP build, all host cores) on a
    bounded sample of the alpha = 1e3 case as the CPU baseline."""
    from paper_1912_12059_gb300 import inputs, nsk

    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    steps = 200
    for alpha in (1e2, 1e3, 1e4):
        wl = inputs.coalescence_2d(alpha=alpha)
        s = nsk.Solver(2, wl.nelem, wl.N, [0.0, 0.0], [1.0, 1.0], 0, nsk.NSK_FP64, stream=stream.cuda_stream)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        U0 = wl.initial_state(s.node_coords())
        s.set_state(U0)
        tpb, fused = pick_schedule(s, args.schedule)
        dt = s.compute_dt(wl.cfl)
        s.step(dt, 3)
        ms = _timed_steps(s, stream, dt, steps)
        gbs = compulsory_bytes(2, 8) * wl.dofs * 5 * steps / (ms / 1e3) / 1e9
        st = s.diagnostics()
        s.close()
        out[f"alpha{alpha:g}"] = {"workload": wl.name, "steps": steps, "dt": dt, "ms_per_step": ms / steps,
                                  "value": wl.dofs * 5 * steps / (ms / 1e3), "unit": "DOF-updates/s",
                                  "dtype": "f64", "schedule": {"tpb": tpb, "fused_face": fused},
                                  "roofline_step_hbm": {"bytes_per_node_stage": compulsory_bytes(2, 8),
                                                        "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                                        "frac": gbs / hbm},
                                  "energy_after": st[1]}
    if not args.no_cpu_baseline:
        rate, desc, thr = oracle_sample(inputs.coalescence_2d(alpha=1e3), target_s=3.0, parallel=True,
                                        ne=(128, 128))
        out["cpu_baseline"] = {"value": rate, "unit": "DOF-updates/s", "cores": thr, "kind": "oracle",
                               "sample": desc}
    return out


def measure_batch_variant(args, n=32, steps=None, with_sequential=True):
    """Batched serving of n uneven 3D collision instances (16^3..48^3 elements, N in {3, 4}, We and
    impact parameter drawn per instance), FP32 operator, autotuned schedule, CUDA-graph replay:
    aggregate DOF-updates/s, the per-step times, and the per-instance step latency p50 / p99 over
    every (step, instance) (time from the step's start until that instance's new state is complete),
    beside the same instances stepped one after another."""
    import torch

    from paper_1912_12059_gb300 import inputs, nsk

    steps = steps or args.steps
    wls = inputs.serving_batch_3d(n, seed=inputs.SEED)
    solvers = []
    for wl in wls:
        s = nsk.Solver(3, wl.nelem, wl.N, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP32_MIXED)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        s.set_state(wl.initial_state(s.node_coords()))
        s.compute_dt(wl.cfl)
        solvers.append(s)
    nodes = sum(s.E * s.npe for s in solvers)
    b = nsk.Batch(solvers)
    tpb, fused, persistent, _ = b.autotune()
    b.step(args.warmup)
    n0 = b.launch_count
    torch.cuda.synchronize()
    step_ms = b.step(steps, timings=True)
    torch.cuda.synchronize()
    launches = b.launch_count - n0
    total_ms = sum(step_ms)
    _, lat = b.step(steps, timings=True, latencies=True)  # the same steps again, with the latency stamps
    flat = np.sort(lat.ravel())
    out = {"workload": f"batched_{n}x_collision3d_E16-48_N3-4", "instances": n, "nodes_total": nodes,
           "dtype": "f32", "steps": steps, "value": nodes * 5 * steps / (total_ms / 1e3), "unit": "DOF-updates/s",
           "ms_per_step": total_ms / steps,
           "schedule": {"tpb": tpb, "fused_face": fused, "kind": BATCH_KINDS[persistent]}, "cuda_graph": b.uses_graph,
           "gpu_launches": launches,
           "step_ms_p50": float(np.percentile(step_ms, 50)), "step_ms_p99": float(np.percentile(step_ms, 99)),
           "per_instance_latency_ms_p50": float(np.percentile(flat, 50)),
           "per_instance_latency_ms_p99": float(np.percentile(flat, 99)),
           "per_instance_latency_ms_max": float(flat[-1])}
    b.close()
    if with_sequential:  # the same instances stepped one after another (no batching)
        seq_ms = 0.0
        for s in solvers:
            s.set_schedule(tpb, fused)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            s.step(s.compute_dt(0.5), 2)
            e1.record()
            torch.cuda.synchronize()
            seq_ms += e0.elapsed_time(e1) / 2
        out["sequential_value"] = nodes * 5 / (seq_ms / 1e3)
    for s in solvers:
        s.close()
    return out


def measure_fp32_variant(args, wl, stream, U0, U64_after, dt, peaks):
    """The FP32 operator (FP64 EoS in the spinodal interval, FP64 dt and sums) on the same workload:
    throughput, HBM roofline of its dominant kernel, and its density L2 error against the FP64 run
    after the same steps from the same initial state."""
    import torch

    from paper_1912_12059_gb300 import nsk

    s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type,
                   nsk.NSK_FP32_MIXED, stream=stream.cuda_stream)
    s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    s.set_state(U0)
    tpb, fused = pick_schedule(s, args.schedule32)
    s.step(dt, args.warmup)
    s.set_profiling(True)
    s.get_profile(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(dt, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.get_profile(reset=True)
    U32 = s.get_state()
    s.close()
    nodes = wl.dofs
    err = float(np.sqrt(((U32[0] - U64_after[0]) ** 2).sum() / (U64_after[0] ** 2).sum()))
    name, (kms, kcnt) = max(prof.items(), key=lambda kv: kv[1][0])
    _, bytes_e = kernel_cost(name, wl.dim, wl.N + 1, 4, traces=trace_fraction(prof), sched=fused)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = bytes_e * wl.n_elem / (kms / max(kcnt, 1) / 1e3) / 1e9
    traffic = MEASURED_TRAFFIC.get((name, 4, wl.n_elem))
    step_gbs = compulsory_bytes(wl.dim, 4) * nodes * 5 * args.steps / (ms / 1e3) / 1e9
    return {"value": nodes * 5 * args.steps / (ms / 1e3), "unit": "DOF-updates/s", "ms_per_step": ms / args.steps,
            "dtype": "f32", "density_l2_rel_err_vs_fp64": err, "steps_compared": args.warmup + args.steps,
            "schedule": {"tpb": tpb, "fused_face": fused},
            # the step on the compulsory bytes (U, K read and written once per stage: 80 B/node in 3D)
            "roofline": {"bound": "hbm", "bytes_per_node_stage": compulsory_bytes(wl.dim, 4), "achieved": step_gbs,
                         "peak": hbm, "unit": "GB/s", "frac": step_gbs / hbm,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
            # the dominant kernel on its own loads and stores (counted from its source)
            "roofline_kernel": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                "frac": achieved / hbm, "traffic": traffic,
                                "traffic_source": TRAFFIC_SOURCE if traffic is not None else None,
                                "bytes_source": "the kernel's own compulsory loads and stores per element"},
            "kernels": {k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1]} for k, v in prof.items()}}


def interface_metrics(U, x):
    """Liquid fraction (nodes with rho above the mean saturation density 1.0634, Sec. 4.2) and the
    distance between the liquid centroids left and right of x = 0.5 (droplet separation)."""
    liquid = U[0] > 1.0634
    left = liquid & (x[0] < 0.5)
    right = liquid & (x[0] >= 0.5)
    xl = float(x[0][left].mean()) if left.any() else float("nan")
    xr = float(x[0][right].mean()) if right.any() else float("nan")
    return {"liquid_fraction": float(liquid.mean()), "separation": xr - xl}


def measure_closure_variant(args):
    """Learned c-closure, 3D collision at 96^3 elements, N=3 (56.6M nodes): network trained on
    (rho, c) element snapshots of FP64 runs of the 64^3 collision at We 10, 40, 80; compared over
    the same simulated time with the explicit FP64 method and the explicit FP32 operator. Returns
    the benchmark line of the closure workload."""
    import torch

    from paper_1912_12059_gb300 import closure, inputs, nsk

    ne_train = args.nelem_train
    ne_eval = args.nelem or 96
    # --- training data: snapshots of explicit FP64 runs ----------------------------------
    t0 = time.perf_counter()
    Xs, Ys = [], []
    for i, we in enumerate((10.0, 40.0, 80.0)):
        wl = inputs.head_on_collision_3d(we=we, nelem=ne_train)
        s = nsk.Solver(3, wl.nelem, 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP64)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        s.set_state(wl.initial_state(s.node_coords()))
        X, Y = closure.collect_snapshots(s, s.compute_dt(wl.cfl), first_step=20, every=10, count=8,
                                         max_per_snapshot=args.samples // 24, rng=np.random.default_rng(i))
        Xs.append(X)
        Ys.append(Y)
        s.close()
    X, Y = torch.cat(Xs), torch.cat(Ys)
    t_data = time.perf_counter() - t0
    perm = torch.randperm(X.shape[0], device=X.device, generator=torch.Generator(device=X.device).manual_seed(0))
    n_val = X.shape[0] // 10
    Xv, Yv, Xt, Yt = X[perm[:n_val]], Y[perm[:n_val]], X[perm[n_val:]], Y[perm[n_val:]]
    wl = inputs.head_on_collision_3d(we=40.0, nelem=ne_eval)
    m = nsk.MLP(2 * (64 + 6), 256, 256, 64, max_batch=4096, max_rows=wl.n_elem)
    m.init_params(seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    closure.train(m, Xt, Yt, steps=args.train_steps, batch=4096, lr=3e-3, lr_min=3e-5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    val_err = closure.validation_error(m, Xv, Yv)

    # --- evaluation at the 96^3 size -----------------------------------------------------
    def timed_run(solver, dt, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        solver.step(dt, n)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    s64 = nsk.Solver(3, wl.nelem, 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP64)
    s64.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    xnodes = s64.node_coords()
    s64.set_state(wl.initial_state(xnodes))
    dt_exp = s64.compute_dt(wl.cfl)
    s64.step(dt_exp, 20)  # c reaches its quasi-equilibrium
    U_start = s64.get_state()
    n_exp = args.eval_steps
    ms64 = timed_run(s64, dt_exp, n_exp)
    U64 = s64.get_state()
    # validation at the evaluation size: network against the explicit FP64 c
    Xe = torch.empty((wl.n_elem, 144), dtype=torch.bfloat16, device="cuda")
    Ye = torch.empty((wl.n_elem, 64), dtype=torch.float32, device="cuda")
    s64.closure_features(Xe)
    s64.closure_targets(Ye)
    val_err_eval = closure.validation_error(m, Xe, Ye)
    s64.close()
    t_end = n_exp * dt_exp

    s32 = nsk.Solver(3, wl.nelem, 3, [0, 0, 0], [1, 1, 1], 0, nsk.NSK_FP32_MIXED)
    s32.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
    s32.set_state(U_start)
    s32.autotune()
    s32.set_state(U_start)
    ms32 = timed_run(s32, dt_exp, n_exp)
    U32 = s32.get_state()
    s32.set_state(U_start)
    s32.set_closure(m, judge_every=10, eta_max=0.5)
    dt_cl = s32.compute_dt(wl.cfl)
    n_cl = int(math.ceil(t_end / dt_cl))
    n0 = s32.launch_count + m.launch_count
    mscl = timed_run(s32, t_end / n_cl, n_cl)
    launches = s32.launch_count + m.launch_count - n0
    st = s32.closure_status()
    Ucl = s32.get_state()
    s32.close()
    m.close()

    def l2(a):
        return float(np.sqrt(((a[0] - U64[0]) ** 2).sum() / (U64[0] ** 2).sum()))

    nodes = wl.dofs
    line = {
        "metric": "DOF-updates/s", "value": nodes * 5 * n_cl / (mscl / 1e3), "unit": "DOF-updates/s",
        "n_gpus": 1, "steps": n_cl, "warmup": 20, "ms_per_step": mscl / n_cl, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": f"learned_closure_3d_E{ne_eval}^3_N3_We40", "nodes": nodes,
                   "train": {"samples": int(X.shape[0]), "source": f"FP64 {ne_train}^3 collision runs, We 10/40/80",
                             "steps": args.train_steps, "batch": 4096, "seconds": t_train, "data_seconds": t_data,
                             "samples_per_s": args.train_steps * 4096 / t_train,
                             "val_rel_err": val_err, "val_rel_err_at_eval_size": val_err_eval},
                   "simulated_time": t_end},
        "closure": {"dt": dt_cl, "steps": n_cl, "wall_ms": mscl, "density_l2_rel_err_vs_fp64": l2(Ucl),
                    "judge_eta": st["eta"], "fallbacks": st["fallbacks"], "interface": interface_metrics(Ucl, xnodes)},
        "explicit_fp64": {"dt": dt_exp, "steps": n_exp, "wall_ms": ms64, "value": nodes * 5 * n_exp / (ms64 / 1e3),
                          "interface": interface_metrics(U64, xnodes)},
        "explicit_fp32": {"dt": dt_exp, "steps": n_exp, "wall_ms": ms32, "value": nodes * 5 * n_exp / (ms32 / 1e3),
                          "density_l2_rel_err_vs_fp64": l2(U32), "interface": interface_metrics(U32, xnodes)},
        "time_to_solution_speedup": {"closure_vs_fp64": ms64 / mscl, "closure_vs_fp32": ms32 / mscl,
                                     "fp32_vs_fp64": ms64 / ms32},
        "gpu_launches": launches,
        "e2e": None, "roofline": None, "cpu_baseline": None,
    }
    return line


def run_closure(args, rank, world):
    """The learned-closure workload (measure_closure_variant) as its own benchmark line."""
    import torch

    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    if rank != 0:
        return 0
    print(json.dumps(measure_closure_variant(args)))
    return 0


def run_gemm(args, rank, world):
    """Tensor-core GEMMs of the closure network's forward pass (BF16 in, FP32 accumulation):
    rows = elements of the evaluation mesh, shapes [rows x 144] . [256 x 144]^T (GELU),
    [rows x 256] . [256 x 256]^T (GELU), [rows x 256] . [64 x 256]^T (store)."""
    import torch

    from paper_1912_12059_gb300 import nsk
    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    rows = args.rows
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((rows, 144), device="cuda", generator=g).to(torch.bfloat16)
    W1 = torch.randn((256, 144), device="cuda", generator=g).to(torch.bfloat16)
    W2 = torch.randn((256, 256), device="cuda", generator=g).to(torch.bfloat16)
    W3 = torch.randn((64, 256), device="cuda", generator=g).to(torch.bfloat16)
    H1 = torch.empty((rows, 256), dtype=torch.bfloat16, device="cuda")
    H2 = torch.empty((rows, 256), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((rows, 64), dtype=torch.float32, device="cuda")
    calls = [("layer1_gelu", lambda: nsk.gemm_bf16(X, W1, epilogue=2, hout=H1), 2 * rows * 144 * 256,
              rows * 144 * 2 + rows * 256 * 2),
             ("layer2_gelu", lambda: nsk.gemm_bf16(H1, W2, epilogue=2, hout=H2), 2 * rows * 256 * 256,
              rows * 256 * 2 * 2),
             ("layer3_store", lambda: nsk.gemm_bf16(H2, W3, epilogue=0, out=Y), 2 * rows * 256 * 64,
              rows * 256 * 2 + rows * 64 * 4)]
    out = {}
    peaks = json.loads(MEASURED_PEAKS.read_text()) if MEASURED_PEAKS.exists() else {}
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    for name, f, flops, nbytes in calls:
        for _ in range(args.warmup):
            assert f() == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"ms": ms, "tflops": flops / ms / 1e9, "frac_of_bf16_peak": flops / ms / 1e9 / tc_peak,
                     "gbs": nbytes / ms / 1e6}
    # the network's inference forward through the library: one fused kernel vs the three GEMMs
    m = nsk.MLP(140, 256, 256, 64, max_batch=4096, max_rows=rows)
    m.init_params(seed=0)
    flops = 2 * rows * (144 * 256 + 256 * 256 + 256 * 64)
    fwd = {}
    # the fused kernel where it applies (warp-specialised, operands by TMA), the fused kernel that runs
    # its stages one after another, and the three per-layer GEMMs
    for name, fused, serial in (("fused", True, 0), ("fused_serial", True, 1), ("three_gemms", False, 0)):
        m.set_fused_forward(fused)
        nsk._test_hook_mlp_fwd_kernel(serial)
        for _ in range(args.warmup):
            m.forward(X, Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            m.forward(X, Y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        fwd[name] = {"ms": ms, "tflops": flops / ms / 1e9,
                     "frac_of_bf16_peak": flops / ms / 1e9 / tc_peak,
                     "hbm_gbs": (rows * 144 * 2 + rows * 64 * 4) / ms / 1e6}
    nsk._test_hook_mlp_fwd_kernel(0)
    m.close()
    if rank == 0:
        ms = fwd["fused"]["ms"]
        print(json.dumps({"metric": "closure MLP forward rows/s", "value": rows / (ms / 1e3), "unit": "rows/s",
                          "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                          "config": {"workload": f"closure_mlp_forward_rows{rows}", "forward": fwd, "layers": out,
                                     "bf16_peak_tflops": tc_peak}}))
    return 0


def run_fp32err(args, rank, world):
    """FP32 operator against FP64 over a long run (the 64^3 collision, We = 40, fixed dt of the
    default bench): density L2 relative error, and each run's mass drift, at checkpoints up to
    --steps steps (5000 when not given)."""
    import torch

    from paper_1912_12059_gb300 import nsk
    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    wl = workload_by_name("collision3d")
    total = args.steps if "--steps" in args.argv else 5000
    solvers = {}
    for prec in (nsk.NSK_FP64, nsk.NSK_FP32_MIXED):
        s = nsk.Solver(wl.dim, wl.nelem, wl.N, list(wl.lo[:wl.dim]), list(wl.hi[:wl.dim]), wl.node_type, prec)
        s.set_params(T=wl.T, kappa=wl.kappa, alpha=wl.alpha, beta=wl.beta, mu=wl.mu)
        solvers[prec] = s
    s64, s32 = solvers[nsk.NSK_FP64], solvers[nsk.NSK_FP32_MIXED]
    U0 = wl.initial_state(s64.node_coords())
    for s in (s64, s32):
        s.set_state(U0)
        s.autotune()
    dt = s64.compute_dt(wl.cfl)
    m0 = {p: s.diagnostics()[0] for p, s in solvers.items()}
    checkpoints = [c for c in (10, 100, 500, 1000, 2000, 5000, 10000, 20000) if c < total] + [total]
    done, rows = 0, []
    t0 = time.time()
    for cp in checkpoints:
        for s in (s64, s32):
            s.step(dt, cp - done)
        done = cp
        r64, r32 = s64.get_state()[0], s32.get_state()[0]
        err = float(np.sqrt(((r32 - r64) ** 2).sum() / (r64 ** 2).sum()))
        rows.append({"steps": cp, "density_l2_rel_err": err,
                     "mass_drift_fp64": (s64.diagnostics()[0] - m0[nsk.NSK_FP64]) / m0[nsk.NSK_FP64],
                     "mass_drift_fp32": (s32.diagnostics()[0] - m0[nsk.NSK_FP32_MIXED]) / m0[nsk.NSK_FP32_MIXED]})
    for s in solvers.values():
        s.close()
    if rank == 0:
        print(json.dumps({"metric": "FP32 density L2 relative error vs FP64", "value": rows[-1]["density_l2_rel_err"],
                          "unit": "relative L2", "n_gpus": 1, "steps": total, "warmup": 0,
                          "higher_is_better": False, "dtype": "f32 vs f64", "data": "synthetic",
                          "config": {"workload": wl.name, "dt": dt, "simulated_time": dt * total,
                                     "wall_s": time.time() - t0, "checkpoints": rows}}))
    return 0


def run_esdirk(args, rank, world):
    """The implicit ESDIRK4 comparison (the esdirk4_implicit variant of the default run) alone; its
    value is the preconditioned 1000x step at the paper's stiff alpha/beta, the explicit run's wall
    time beside it."""
    import torch

    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    stream = torch.cuda.Stream()
    v = measure_esdirk_variant(args, stream)
    if rank == 0:
        st = v["stiff_paper_parameters"]
        x = st["esdirk4_1000x_block_precond"]
        print(json.dumps({"metric": "wall ms to the simulated time of 1000 explicit LSRK4 steps (one implicit ESDIRK4 "
                                    "step at 1000x the explicit dt, element-block preconditioner, alpha 1e3, beta 1e-3)",
                          "value": x["wall_ms"], "unit": "ms", "n_gpus": 1, "steps": x["steps"], "warmup": 0,
                          "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                          "explicit_wall_ms": st["explicit_lsrk4"]["wall_ms"], "config": v}))
    return 0


def run_riemann1d(args, rank, world):
    """The 1D sharp-interface Riemann problem with FV sub-cell shock capturing alone (the
    riemann1d_subcell variant of the default run as its own line)."""
    import torch

    from paper_1912_12059_gb300.build import build_library

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build_library()
    stream = torch.cuda.Stream()
    v = measure_subcell_variant(args, stream)
    if rank == 0:
        t = v["time_to_solution"]
        print(json.dumps({"metric": "DOF-updates/s", "value": t["value"], "unit": "DOF-updates/s", "n_gpus": 1,
                          "steps": t["steps"], "warmup": 0, "ms_per_step": t["ms_per_step"], "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic", "config": v}))
    return 0


def run_fp64peak(args, rank, world):
    """The FMA throughput probe alone (nsk_measure_fma_rate): FP64 and FP32 FMA rates of this GPU
    with the SM clock sampled during the launches, beside the peaks derived from the SM count, the
    FMAs per SM and clock and the sampled clock (the ALU roofline denominator of the FP64 path)."""
    import torch

    from paper_1912_12059_gb300 import nsk
    from paper_1912_12059_gb300.build import build_library

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build_library()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    res = {}
    for prec, tag, iters in ((nsk.NSK_FP64, "fp64", 1 << 17), (nsk.NSK_FP32_MIXED, "fp32", 1 << 20)):
        with ClockSampler(local) as clk:
            for _ in range(args.warmup):
                nsk.measure_fma_rate(prec, iters=iters // 8)
            runs = [nsk.measure_fma_rate(prec, iters=iters) for _ in range(args.steps)]
        c = clk.summary()
        best = max(r[0] for r in runs)
        mhz = c["sm_mhz"] or 2070.0
        derived = alu_peak_tflops(sms, mhz, fp64=(tag == "fp64"))
        res[tag] = {"tflops_best": best, "tflops_median": statistics.median(r[0] for r in runs),
                    "launch_ms_median": statistics.median(r[1] for r in runs), "sm_mhz_median": c["sm_mhz"],
                    "sm_max_mhz": c["sm_max_mhz"], "clock_reasons": c["reasons"],
                    "derived_at_sampled_clock": derived, "measured_over_derived": best / derived,
                    "fma_per_sm_clk_measured": best * 1e12 / (2 * sms * mhz * 1e6)}
    if rank == 0:
        print(json.dumps({"metric": "FP64 FMA throughput", "value": res["fp64"]["tflops_best"], "unit": "TFLOP/s",
                          "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "fma_rate_probe", "sms": sms,
                                     "launch": "8 blocks x 256 threads per SM, 8 independent FMA chains per thread"},
                          "fp64": res["fp64"], "fp32": res["fp32"]}))
    return 0


def make_parser():
    """The command line of the benchmark."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="collision3d",
                    choices=["collision3d", "coalescence2d", "interface1d", "batch", "closure", "gemm", "riemann1d",
                             "fp32err", "esdirk", "fp64peak"])
    ap.add_argument("--rows", type=int, default=884736, help="gemm: rows (elements)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variants of the default run (FP32, HLLC, original NSK, sub-cell, ESDIRK4)")
    ap.add_argument("--nelem-train", type=int, default=64, help="closure: training mesh (elements per direction)")
    ap.add_argument("--samples", type=int, default=200000, help="closure: training samples")
    ap.add_argument("--train-steps", type=int, default=4000, help="closure: Adam steps")
    ap.add_argument("--eval-steps", type=int, default=100, help="closure: explicit steps of the comparison")
    ap.add_argument("--batch", type=int, default=32, help="instances of the batch workload")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nelem", type=int, default=0, help="override elements per direction (profiling runs)")
    ap.add_argument("--schedule", default="", help='fixed stage schedule "TPB,FUSED" instead of the autotuner')
    ap.add_argument("--schedule32", default="", help='the same for the FP32 variant')
    return ap


def main(argv=None):
    argv = sys.argv[1:] if argv is None else list(argv)
    args = make_parser().parse_args(argv)
    args.argv = argv  # the flags given explicitly (some workloads default differently without them)
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "closure":
        return run_closure(args, rank, world)
    if args.workload == "gemm":
        return run_gemm(args, rank, world)
    if args.workload == "riemann1d":
        return run_riemann1d(args, rank, world)
    if args.workload == "fp32err":
        return run_fp32err(args, rank, world)
    if args.workload == "esdirk":
        return run_esdirk(args, rank, world)
    if args.workload == "fp64peak":
        return run_fp64peak(args, rank, world)
    if args.workload == "batch":
        if args.precision == "fp64" and "--precision" not in argv:
            args.precision = "fp32"
        return run_batch(args, rank, world)
    wl = workload_by_name(args.workload)
    if args.nelem:
        import dataclasses

        wl = dataclasses.replace(wl, nelem=(args.nelem,) * wl.dim, name=f"{wl.name}_resized_E{args.nelem}")
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    try:
        return run_gpu(args, wl, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
