"""Benchmark of the ADI heat step on the 2048 x 4096 five-region cell.

Workload: the layered cryogenic cell of the paper's Fig. "object" on a
2048 (r) x 4096 (z) grid, seeded log-uniform conductivities, uniform heat
capacities and heater source, dt = 50 x the explicit stability limit; one
bench step = one ADI time step (r-sweep + z-sweep).  The FP32 path is the
headline (`value`); the FP64 path is measured side by side.

Timing: W untimed warm-up steps, then K steps, each preceded by an L2 flush
(a 512 MB device write) and bracketed by CUDA events on the solver's stream,
with an event between the two sweeps for per-kernel durations.
`value` = active cells x K / (sum of step times).  `e2e` runs the same job
through the C ABI with host buffers: upload of the initial field, K steps,
download of the result, timed as a whole.  `ensemble` times the 512-member
batched ensemble (500 graph-replayed steps under the autotuned schedule).

--impl reference times the FP64 CPU oracle (the method's plain restatement,
OpenMP over lines as in the paper's Sec. 4) on a bounded number of steps of
the same workload.  Multi-GPU (torchrun): every rank runs an independent
replica (the single-domain solve does not shard); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import heat as H  # noqa: E402

METRIC = "cell-steps/s vs HBM roofline"
UNIT = "cell-steps/s"
WORKLOAD = "config2: five-region layered cell 2048x4096, seed 2, dt=50*tau_exp"
ELEM = {"fp64": 8, "fp32": 4}
# Algorithmic FP64 flops per cell and sweep of the literal form (the FP64
# path): right-hand side w T + A-(T_- - T) + A+(T_+ - T) + q (2 sub, 3 fma,
# 1 add = 9), forward recurrence d' = d inv + f d'_prev (mul + fma = 3),
# backward x = d' + cp x_next (fma = 2).  FMA counts as 2 flops.
FP64_FLOPS_PER_CELL_SWEEP = 14
# GB300's nominal FP64 rate (not measured on this machine; MEASURED_PEAKS.json
# has HBM and BF16 only).
FP64_NOMINAL_TFLOPS = 1.25
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def csrc_sha() -> str:
    """sha256 (16 hex) of the CUDA/C++ sources the heat kernels are built from
    (the heat_* files: the surrogate's sources do not change them)."""
    import hashlib
    d = os.path.join(ROOT, "paper_1912_03744_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.startswith("heat_") and f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM bytes (read + write) per launch, keyed (kernel, precision, Nr, Nz),
    from the committed ncu summary profiles/traffic.txt.  The summary records
    the source hash of the kernels it measured; when the sources have changed
    since, the numbers no longer describe these kernels and none are used."""
    out, sha = {}, None
    if not os.path.exists(TRAFFIC_FILE):
        return out, "no traffic summary"
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if len(f) >= 2 and f[0] == "csrc_sha":
            sha = f[1]
        elif len(f) == 5 and not line.startswith("#") and f[0] != "kernel":
            out[(f[0], f[1], int(f[2]), int(f[3]))] = float(f[4])
    if sha != csrc_sha():
        return {}, "kernel sources changed since the capture in profiles/traffic.txt"
    return out, "profiles/traffic.txt"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            # every 20 ms (the headline's timed region lasts a fraction of a
            # second), started before the region so that it samples within it
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.p = None
        self.t0 = time.time()  # samples count from here to __exit__
        return self

    def __exit__(self, *a):
        self.rows = []
        t1 = time.time()
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        import datetime
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                t = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                t = None
            if t is None or self.t0 <= t <= t1:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce_max(x, ws):
    """The maximum of x over the ranks (the replicas' slowest time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _reduce_sum(x, ws):
    """The sum of x over the ranks."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_members(cells, ws):
    """Members of an ensemble dealt to ws ranks with balanced cell counts:
    largest first, each to the rank with the fewest cells so far (ties to the
    lowest rank); deterministic, every member on exactly one rank, each
    rank's list in ascending member order."""
    load = [0] * ws
    out = [[] for _ in range(ws)]
    for i in sorted(range(len(cells)), key=lambda i: (-cells[i], i)):
        r = min(range(ws), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += cells[i]
    return [sorted(o) for o in out]


def _whole_job(units_per_rank, ws, max_seconds):
    """Whole-job throughput of ws replicas that each processed units_per_rank
    units, over the slowest rank's time (weak scaling)."""
    return ws * units_per_rank / max_seconds


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def time_gpu(p, precision, steps, warmup, flush):
    """Per-step CUDA-event timing with an L2 flush before each step: `steps`
    whole steps (an event pair around each) give the step time; as many more
    with an event between the two sweeps give each sweep's time (that event
    takes away the overlap of the r-sweep's end with the z-sweep's start, about
    a microsecond of a step)."""
    import torch
    from paper_1912_03744_gb300 import HeatSolver
    probe = HeatSolver(p, 1.0, precision=precision)
    tau = H.DT_FACTOR * probe.tau_exp
    probe.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = HeatSolver(p, tau, precision=precision, stream=stream)
        s.step(warmup)
        n = steps
        es = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n):
            flush.zero_()
            es[k][0].record(stream)
            s.sweep(0)
            s.sweep(1)
            es[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            s.sweep(0)
            ev[k][1].record(stream)
            s.sweep(1)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    step_ms = [es[k][0].elapsed_time(es[k][1]) for k in range(n)]
    r_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(n)]
    z_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(n)]
    E, Phi, Q = s.energy()
    launches = s.launches_per_step() * n
    s.close()
    return dict(tau=tau, step_ms=step_ms, r_ms=r_ms, z_ms=z_ms, wall=wall, launches=launches, E=E)


def time_e2e(p, precision, steps):
    """One job through the C ABI with host buffers: upload, K steps, download."""
    import torch
    from paper_1912_03744_gb300 import HeatSolver
    probe = HeatSolver(p, 1.0, precision=precision)
    tau = H.DT_FACTOR * probe.tau_exp
    probe.close()
    s = HeatSolver(p, tau, precision=precision)
    T0 = np.full((p.Nz, p.Nr), p.T_init)
    s.set_field(T0)
    s.step(2)
    s.field()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_field(T0)
    s.step(steps)
    out = s.field()
    t1 = time.perf_counter()
    s.close()
    assert np.isfinite(out).all()
    nbytes = p.Nr * p.Nz * ELEM[precision]
    return t1 - t0, nbytes


def active_cells(solver, p):
    """Cells whose centre (from the library's grid) lies in a region box."""
    rc, zc = solver.centres()
    act = np.zeros((len(zc), len(rc)), dtype=bool)
    for (r0, r1, z0, z1) in np.asarray(p.boxes, dtype=np.float64).reshape(-1, 4):
        act |= ((zc >= z0) & (zc <= z1))[:, None] & ((rc >= r0) & (rc <= r1))[None, :]
    return int(act.sum())


def time_config1(steps=200, warmup=10):
    """Config 1: the 64 x 128 five-region cell in FP64, 200 steps at
    dt = 50 tau_exp; CUDA events around the 200 steps on the solver's stream.
    The 64 KB field lives in L2 (and would fit one SM's shared memory), so
    this is a latency figure, reported in microseconds per step."""
    import torch
    from paper_1912_03744_gb300 import HeatSolver
    p = H.config1()
    probe = HeatSolver(p, 1.0, precision="fp64")
    tau = H.DT_FACTOR * probe.tau_exp
    act = active_cells(probe, p)
    probe.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = HeatSolver(p, tau, precision="fp64", stream=stream)
        s.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = s.launches_per_step()
        s.close()
    return {"workload": "config1: five-region cell 64x128, seed 0, dt=50*tau_exp", "precision": "fp64",
            "steps": steps, "us_per_step": 1e3 * ms / steps, "cell_steps_per_s": act * steps / (ms * 1e-3),
            "active_cells": act, "launches_per_step": launches, "bound": "latency",
            "note": "64 KB field, resident in L2: the HBM roofline does not apply"}


def time_full_method(window_steps=None):
    """The paper's full method (temperature-dependent laws, simple iteration,
    adaptive tau, erf-smoothed pulsed source) on its example shape: the graded
    1210 x 100 grid without terminal cap, t_per 0.1 s, t_src 0.01 s, t_trs
    1e-4 s, the per-step estimates t_src/100 and t_trs/1000, synthetic laws.
    Timed: the window from 3 base steps before the first switch-off through
    its transition (1000 steps of t_trs/1000) and 5 base steps after it, the
    stretch where the method takes most of its steps per period; wall time
    of heat_nl_advance (it synchronizes once per batch of iterations)."""
    import torch
    from paper_1912_03744_gb300 import HeatNl
    p, m = H.paper_example_nl()
    m.j2 = m.j2 * 4e3
    kw = dict(eps=1e-9, s_max=20, tau_base=m.t_src / 100, tau_trs=m.t_trs / 1000, tau_min=1e-12)
    s = HeatNl(p, m, **kw)
    s.set_time(0.0)
    s.advance(2e-5)  # warm-up: 200 transition steps
    t0 = m.t_src - 3 * kw["tau_base"]
    t_end = m.t_src + m.t_trs + 5 * kw["tau_base"]
    s.set_time(t0)
    torch.cuda.synchronize()
    l0 = s.launches()
    w0 = time.perf_counter()
    st = s.advance(t_end)
    w = time.perf_counter() - w0
    launches = s.launches() - l0
    T = s.field()
    s.close()
    cells = p.Nr * p.Nz
    its = st["iters1"] + st["iters2"]
    return {"workload": "paper example shape: graded 1210x100, no cap, erf pulse t_per 0.1 s, t_src 0.01 s, "
                        "t_trs 1e-4 s, synthetic T-dependent laws, FP64",
            "window_s": [t0, t_end], "steps": st["steps"], "halvings": st["halvings"],
            "iterations_per_half_step": its / (2 * st["steps"]), "wall_s": w, "steps_per_s": st["steps"] / w,
            "cell_steps_per_s": cells * st["steps"] / w, "cell_iterations_per_s": cells * its / w,
            "launches": launches, "finite": bool(np.isfinite(T).all()),
            "stored_cells": 80 * 1210 + 20 * 800,
            "bound": "latency: 100 r-lines and 1210 z-lines of FP64 line solves per iteration, a host read of the "
                     "convergence slots per batch of iterations"}


def step_roofline(cells_active, word, ms_per_step):
    """Whole-step algorithmic bandwidth (read + write of every active cell in
    each of the two sweeps) against the measured copy bandwidth."""
    peak, kind = _peaks()
    b = 4 * word * cells_active
    ach = b / (ms_per_step * 1e-3) / 1e9
    return {"kernel": "whole step", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": None, "algorithmic_bytes": b, "peak_kind": kind, "cells": "active"}


def time_ensemble(steps, warmup, precision="fp32", tuning=None, rank=0, ws=1):
    """The 512-member batched ensemble (Nr 64..512, Nz 128..1024, jittered
    layers and materials), dt = 50 x each member's explicit limit, autotuned
    schedule, graph-replayed steps; CUDA events on the caller's stream around
    all timed steps.  The two field buffers (~0.7 GB in FP32) exceed L2.
    With ws ranks the members are sharded over them by cell count
    (shard_members: the ensemble's members are independent problems, so no
    data crosses ranks); the time is the slowest rank's, the work all
    ranks' (strong scaling of the fixed ensemble)."""
    import torch
    from paper_1912_03744_gb300 import HeatBatch
    probs = H.config3_members(512)
    n_all = len(probs)
    if ws > 1:
        probs = [probs[i] for i in shard_members([q.Nr * q.Nz for q in probs], ws)[rank]]
    t0 = time.perf_counter()
    b = HeatBatch(probs, [1.0] * len(probs), precision=precision)
    b.set_dt([H.DT_FACTOR * m.tau_exp for m in b.members])
    create_s = time.perf_counter() - t0
    act = sum(active_cells(m, p) for m, p in zip(b.members, probs))
    if tuning is None:
        tune_ms = b.tune(trial_steps=3)
    else:
        b.set_tuning(*tuning)
        tune_ms = None
    b.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    b.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ok = all(np.isfinite(b.members[i].field()).all() for i in (0, len(probs) // 2, len(probs) - 1))
    cells = b.cells
    if ws > 1:
        ms = _reduce_max(ms, ws)
        act = int(_reduce_sum(act, ws))
        cells = int(_reduce_sum(cells, ws))
        ok = _reduce_sum(0.0 if ok else 1.0, ws) == 0.0
    out = {"workload": "config3: 512-member ensemble, Nr U{64..512}, Nz U{128..1024}, seed 3, dt=50*tau_exp",
           "precision": precision, "members": n_all, "cells": cells, "active_cells": act,
           "sharding": f"members over {ws} ranks by cell count" if ws > 1 else "one rank",
           "steps": steps, "ms_per_step": ms / steps, "cell_steps_per_s": act * steps / (ms * 1e-3),
           "member_steps_per_s": n_all * steps / (ms * 1e-3),
           "fields_per_s_500_steps": n_all / (500 * ms / steps * 1e-3),
           "tuning": dict(zip(("rK", "band", "zwpb"), b.tuning())), "tune_ms_per_step": tune_ms,
           "launches_per_step": b.launches_per_step(), "graph_replay": True, "create_s": create_s,
           "finite": bool(ok), "l2": "inputs larger than L2",
           "roofline": step_roofline(act, ELEM[precision], ms / steps)}
    b.close()
    return out


def time_config4(steps, warmup, grid=(8192, 16384)):
    """Precision stress at full size: 8192 x 16384 (134 M cells), conductivity
    contrast 1e4, FP32 line solves with the residual refinement (the residual
    from the FP64 coefficients in extended precision); CUDA
    events around `steps` steps (each field is 537 MB, larger than L2), and
    the FP64 heat balance of one step measured by the library itself:
    E(next) - E(now) - tau Q - tau/2 (Phi(now) + Phi(next)), relative to the
    energy change.  Accuracy against the FP64 oracle is the 1024 x 2048
    subsample test (tests/test_gpu_parity.py)."""
    import torch
    from paper_1912_03744_gb300 import HeatSolver
    p = H.config4(*grid)
    probe = HeatSolver(p, 1.0, precision="fp32_refined")
    tau = H.DT_FACTOR * probe.tau_exp
    act = active_cells(probe, p)
    probe.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = HeatSolver(p, tau, precision="fp32_refined", stream=stream)
        s.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        E0, Phi0, Q = s.energy()
        s.step(1)
        E1, Phi1, _ = s.energy()
        launches = s.launches_per_step()
        s.close()
    resid = (E1 - E0) - tau * Q - 0.5 * tau * (Phi0 + Phi1)
    return {"workload": f"config4: {p.Nr}x{p.Nz}, k 0.04/400 (contrast 1e4), seed 4, dt=50*tau_exp",
            "precision": "fp32_refined", "steps": steps, "ms_per_step": ms / steps,
            "cell_steps_per_s": act * steps / (ms * 1e-3), "active_cells": act,
            "heat_balance_rel": abs(resid) / abs(E1 - E0), "launches_per_step": launches,
            "roofline": step_roofline(act, 4, ms / steps),
            "accuracy": "1024x2048 subsample vs FP64 oracle: tests/test_gpu_parity.py::test_config4_subsample_against_the_oracle",
            "l2": "inputs larger than L2"}


SURR_WEIGHTS = os.path.join(ROOT, "paper_1912_03744_gb300", "weights", "fno_config5.npy")


def time_surrogate(n_train, epochs, n_eval=512, n_infer=4096, tols=(0.01, 0.05), n_check=8, batch=64):
    """Config 5: the FNO surrogate (128 x 256 grid, width 32, 12 x 12 modes, 4
    layers) of the field after 2000 ADI steps at a fixed dt.  The network is
    the committed trained one (paper_1912_03744_gb300/weights, written by
    train_surrogate.py; its training summary is beside it) or, without that
    file, one trained here on n_train solver runs for `epochs` passes.  Its
    rise-relative max error is measured on n_eval fresh solver runs (a seed
    used by no training run); fields/s of the plain solver (with and without
    its per-call setup), of the network alone and of the solver-checked
    inference (n_check members re-solved, fallback to the solver for the
    whole batch when one exceeds tol) on the same n_infer parameter sets."""
    import torch
    from paper_1912_03744_gb300 import HeatBatch, HeatSolver, Surrogate
    from workloads import fno as F
    D = F.FnoDims()
    ref = H.config5_reference_problem()
    probe = HeatSolver(ref, 1.0, precision="fp64")
    dt = H.DT_FACTOR * probe.tau_exp
    probe.close()
    pev = H.config5_params(n_eval, seed=7)
    pin = H.config5_params(n_infer, seed=8)
    s = Surrogate(H.config5_problem(pev[0]), D, heater=H.HEATER, dt=dt, steps=2000, max_batch=batch)
    cells = D.Nz * D.Nr
    out = {"workload": "config5: FNO 128x256, width 32, 12x12 modes, 4 layers, horizon 2000 steps",
           "n_eval": n_eval, "n_infer": n_infer, "n_check": n_check, "n_params": s.n_params}
    if os.path.exists(SURR_WEIGHTS):
        s.set_params(np.load(SURR_WEIGHTS).astype(np.float32))
        meta = os.path.splitext(SURR_WEIGHTS)[0] + ".json"
        out["network"] = {"weights": os.path.relpath(SURR_WEIGHTS, ROOT),
                          "training": json.load(open(meta)) if os.path.exists(meta) else None}
    else:
        ptr = H.config5_params(n_train, seed=5)
        s.set_params(F.init_params(D, 7).astype(np.float32))
        data = torch.empty((n_train, D.Nz, D.Nr), dtype=torch.float32, device="cuda")
        s.solve(ptr, out=data)
        t0 = time.perf_counter()
        loss = s.train(ptr, data, epochs=epochs, batch=batch, lr=1e-3, lr_min_frac=0.02, seed=1)
        torch.cuda.synchronize()
        out["network"] = {"trained_here": {"n_train": n_train, "epochs": epochs, "final_loss": loss,
                                           "train_s": time.perf_counter() - t0}}
        del data
    ev = torch.empty((n_eval, D.Nz, D.Nr), dtype=torch.float32, device="cuda")
    s.solve(pev, out=ev)
    err = s.errors(pev, ev)
    del ev
    out["eval_err"] = {"p50": float(np.percentile(err, 50)), "p90": float(np.percentile(err, 90)),
                       "p99": float(np.percentile(err, 99)), "max": float(err.max()),
                       "frac_le_1pct": float(np.mean(err <= 0.01)), "frac_le_5pct": float(np.mean(err <= 0.05))}
    T = torch.empty((n_infer, D.Nz, D.Nr), dtype=torch.float32, device="cuda")
    s.forward(pin[:batch], out=T[:batch])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.solve(pin, out=T)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.forward(pin, out=T)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t0
    checked = {}
    for tol in tols:
        t0 = time.perf_counter()
        _, used, cerr = s.infer_checked(pin, n_check=n_check, tol=tol, seed=3, out=T)
        torch.cuda.synchronize()
        t_chk = time.perf_counter() - t0
        checked[f"tol_{tol:g}"] = {"fields_per_s": n_infer / t_chk, "used_fallback": used, "max_checked_err": cerr,
                                   "gain_over_solver": t_solve / t_chk}
    s.close()
    # the plain batched solver without its per-call setup: 512 members of the
    # same cell, 2000 graph-replayed steps
    nb = 512
    b = HeatBatch([H.config5_problem(x) for x in pin[:nb]], [dt] * nb, precision="fp32")
    b.step(10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(2000)
    b.sync()
    t_steps = time.perf_counter() - t0
    b.close()
    out["fields_per_s"] = {"solver": n_infer / t_solve, "solver_steps_only": nb / t_steps,
                           "network": n_infer / t_net}
    out["checked"] = checked
    out["solver_cell_steps_per_s"] = n_infer * cells * 2000 / t_solve
    return out


def cpu_baseline(p, budget_s=12.0, max_steps=50, warmup=1):
    """The FP64 oracle as it stands, all host cores, bounded number of steps
    after `warmup` untimed ones."""
    import oracle
    from oracle import Oracle
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    cores = oracle.max_threads()
    for _ in range(warmup):
        o.step(tau, 1)
    n = 0
    t0 = time.perf_counter()
    while n < max_steps and (time.perf_counter() - t0) < budget_s:
        o.step(tau, 1)
        n += 1
    dt = time.perf_counter() - t0
    return n, dt, cores


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    p = H.config2()
    from oracle import Oracle
    act = int((Oracle(p).grid()["region"] >= 0).sum())
    # K steps of about 40 ms each on the host cores, capped at two minutes
    n, dt, cores = cpu_baseline(p, budget_s=min(120.0, max(5.0, 0.5 * args.steps)), max_steps=max(1, args.steps),
                                warmup=args.warmup)
    v = act * n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * dt / n, "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [p.Nr, p.Nz], "precision": "fp64", "solver": "cpu oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n} steps of the full 2048x4096 workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-main", action="store_true",
                    help="time the headline path only (no side-by-side, e2e or CPU legs); for profiling")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-steps", type=int, default=500)
    ap.add_argument("--ensemble-only", action="store_true", help="time the ensemble leg only; for profiling")
    ap.add_argument("--ensemble-tuning", default=None,
                    help="K,band,zwpb: fixed ensemble schedule instead of the autotuner")
    ap.add_argument("--no-config4", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-train", type=int, default=4096, help="solver runs the surrogate trains on")
    ap.add_argument("--surrogate-epochs", type=int, default=10)
    ap.add_argument("--config4-steps", type=int, default=20)
    ap.add_argument("--config4-grid", default="8192,16384", help="Nr,Nz of the config-4 leg (profiling: smaller)")
    ap.add_argument("--leg", default=None, choices=["config1", "config4", "ensemble", "surrogate", "full"],
                    help="time one leg only and print it (for profiling)")
    ap.add_argument("--nr", type=int, default=2048)
    ap.add_argument("--nz", type=int, default=4096)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()

    ens_tuning = tuple(int(x) for x in args.ensemble_tuning.split(",")) if args.ensemble_tuning else None
    if args.leg:
        legs = {"config1": lambda: time_config1(),
                "config4": lambda: time_config4(args.config4_steps, args.warmup,
                                                tuple(int(x) for x in args.config4_grid.split(","))),
                "ensemble": lambda: time_ensemble(args.ensemble_steps, args.warmup, tuning=ens_tuning),
                "surrogate": lambda: time_surrogate(args.surrogate_train, args.surrogate_epochs),
                "full": lambda: time_full_method()}
        print(json.dumps({"leg": args.leg, **legs[args.leg]()}), flush=True)
        return
    if args.ensemble_only:
        print(json.dumps({"ensemble_only": True, **time_ensemble(args.ensemble_steps, args.warmup,
                                                                 tuning=ens_tuning)}), flush=True)
        return
    p = H.config2(args.nr, args.nz)
    from paper_1912_03744_gb300 import HeatSolver
    probe = HeatSolver(p, 1.0, precision="fp64")
    act = active_cells(probe, p)
    probe.close()
    ncell = p.Nr * p.Nz
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    other = "fp64" if args.precision == "fp32" else "fp32"

    _barrier(ws)
    with Clocks(local) as clk:
        main_t = time_gpu(p, args.precision, args.steps, args.warmup, flush)
    if args.only_main:
        tot = sum(main_t["step_ms"])
        print(json.dumps({"only_main": True, "ms_per_step": tot / args.steps,
                          "rsweep_ms": statistics.mean(main_t["r_ms"]),
                          "zsweep_ms": statistics.mean(main_t["z_ms"])}), flush=True)
        return
    side_steps = max(3, min(args.steps, 200))
    side_t = time_gpu(p, other, side_steps, args.warmup, flush)
    e2e_s, e2e_bytes = time_e2e(p, args.precision, args.steps)
    c1 = time_config1()
    full = time_full_method()
    ens = None if args.no_ensemble else time_ensemble(args.ensemble_steps, args.warmup, tuning=ens_tuning,
                                                      rank=rank, ws=ws)
    c4 = None if args.no_config4 else time_config4(args.config4_steps, args.warmup)
    surr = None if args.no_surrogate else time_surrogate(args.surrogate_train, args.surrogate_epochs)
    _barrier(ws)

    tot_ms = sum(main_t["step_ms"])
    tot_ms = _reduce_max(tot_ms, ws)
    e2e_s = _reduce_max(e2e_s, ws)
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = _peaks()
    value = _whole_job(act * args.steps, ws, tot_ms * 1e-3)

    traffic, traffic_src = load_traffic()

    def roof(t, precision):
        """The dominant kernel is the r-sweep, one launch per step (the longest
        single kernel of the step; the z-sweep is three shorter launches,
        reported beside it as a group).  Algorithmic bytes: read and write of
        every active cell once per sweep.  The FP64 path is bound by GB300's
        FP64 units, so its line carries the FP64 flop rate against the nominal
        FP64 peak as well."""
        r_avg = statistics.mean(t["r_ms"])
        z_avg = statistics.mean(t["z_ms"])
        bytes_launch = 2 * ELEM[precision] * act
        ach = bytes_launch / (r_avg * 1e-3) / 1e9
        zach = bytes_launch / (z_avg * 1e-3) / 1e9
        out = {"kernel": "rsweep", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
               "frac": ach / peak, "traffic": traffic.get(("rsweep", precision, p.Nr, p.Nz)),
               "traffic_source": traffic_src,
               "algorithmic_bytes": bytes_launch, "peak_kind": peak_kind, "cells": "active",
               "rsweep_ms": r_avg, "zsweep_ms": z_avg,
               "zsweep_group": {"achieved": zach, "frac": zach / peak, "launches": 3,
                                "traffic": traffic.get(("zsweep", precision, p.Nr, p.Nz))}}
        if precision == "fp64":
            fl = FP64_FLOPS_PER_CELL_SWEEP * act
            out["alu"] = {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_NOMINAL_TFLOPS, "peak_kind": "nominal",
                          "flops_per_cell_sweep": FP64_FLOPS_PER_CELL_SWEEP,
                          "rsweep_achieved": fl / (r_avg * 1e-3) / 1e12,
                          "rsweep_frac": fl / (r_avg * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS,
                          "zsweep_achieved": fl / (z_avg * 1e-3) / 1e12,
                          "zsweep_frac": fl / (z_avg * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS}
        return out

    side_ms = sum(side_t["step_ms"]) / len(side_t["step_ms"])
    cpu = None
    if not args.no_cpu_baseline:
        n, dt, cores = cpu_baseline(p)
        cpu = {"value": act * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} steps of the full {p.Nr}x{p.Nz} workload"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [p.Nr, p.Nz], "precision": args.precision,
                   "active_cells": act, "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"replicas x{ws}"},
        "roofline": roof(main_t, args.precision),
        "cpu_baseline": cpu,
        "e2e": {"value": _whole_job(act * args.steps, ws, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": e2e_bytes / args.steps, "d2h_bytes_per_step": e2e_bytes / args.steps},
        "gpu_launches": main_t["launches"],
        "clocks": clk.summary(),
        "config1": c1,
        "full_method": full,
        "ensemble": ens,
        "config4": c4,
        "surrogate": surr,
        "side_by_side": {other: {"value": act / (side_ms * 1e-3), "ms_per_step": side_ms,
                                 "steps": len(side_t["r_ms"]), "roofline": roof(side_t, other)}},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
