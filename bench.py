"""Benchmark: LLG cell-steps/s of the full H_eff + Euler step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl grace|reference]
                    [--workload block|film_large|film_small]

The headline workload is the 256x256x64 block (4.19 M cells of 3 nm, padded grid
512x512x128), the largest single-GPU configuration.  One "step" is one pass of the hot
path over it: the demag convolution (x C2R, y FFT, z FFT with the tensor product, and
their inverses), exchange, anisotropy, Zeeman, explicit Euler with renormalisation and
the x R2C of the new state (four kernels per step on this split path; films of at most
four cells in z take two).  Inputs are resident in HBM when the timed region starts;
every timed step is preceded by an L2 flush (a 256 MiB write), so no step finds the
previous one's data in the 129 MB L2.

For N > 1 (torchrun, one process per GPU) every rank steps its own replica of the film
(replicas only: the workload has no data exchange), value = all ranks' cell-steps / the
slowest rank's time.  ``--impl reference`` times the FP64 CPU oracle (the only reference
implementation: the paper's own code is not available) on rank 0, one single-threaded
replica of the film per host core.

Beside the headline the line carries the dominant kernel's HBM roofline, the whole step
against the same peak, end-to-end throughput from host buffers, the oracle on one and on
all host cores, the SM clocks sampled during the timed loop, and (unless ``--no-extras``)
the 1024x256x4 film with its own rooflines, the 256-film ensemble, the adjoint's forward
and backward rates at its stated 4,096 steps, the paper-shaped cube sweep and a
vendor-FFT demag comparison.  ``--profile-run NAME`` only takes plain-launch steps of a
workload, for ncu.

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LLG cell-steps/s on 1 GB300 (full H_eff + step), % HBM roofline, vs oracle"
UNIT = "cell-steps/s"
L2_FLUSH_BYTES = 256 << 20
E2E_HANDLES = 4           # handles (and streams) taking the end-to-end steps in turn


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="grace", choices=["grace", "reference"])
    ap.add_argument("--workload", default="block", choices=["block", "film_large", "film_small"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=-1,
                    help="oracle replicas for the all-cores CPU figure (-1: every host core, 0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the block / ensemble / adjoint measurements")
    ap.add_argument("--profile-run", default=None,
                    choices=["film_large", "block", "film_small", "adjoint_film", "ensemble",
                             "ensemble_persistent"],
                    help="no measurement: take --steps plain-launch steps of this workload (for ncu)")
    return ap.parse_args()


def profile_run(name, steps):
    """Plain launches (no graphs) of `steps` steps, so that a profiler sees every kernel.
    ensemble: the 256-film batch (ensemble_persistent: the same batch in one persistent
    launch); adjoint_film: `steps` forward steps keeping checkpoints every 16, then the
    discrete adjoint of those steps from them."""
    import numpy as np
    import torch
    import workloads
    from paper_1411_2565_gb300 import _lib
    from paper_1411_2565_gb300.build import build
    from paper_1411_2565_gb300.grace import Grace, GraceBatch
    build()
    persistent = name == "ensemble_persistent"
    if persistent:
        name = "ensemble"
    w = getattr(workloads, name)()
    opts = {_lib.OPT_GRAPH: 0}
    if name == "ensemble":
        if persistent:
            opts[_lib.OPT_PERSISTENT] = 1      # one cooperative launch per call
        g = GraceBatch(w.films, device="cuda:0", options=opts)
        g.set_m(torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).cuda())
        g.step(steps, w.dt)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": name, "steps": steps}), flush=True)
        return
    f, m0 = w.films[0], w.m0[0]
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device="cuda:0", options=opts)
    g.set_hext(f.hext)
    if getattr(w, "ms_field", None) is not None:
        g.set_ms_field(torch.from_numpy(w.ms_field.reshape(-1)).cuda())
    if name == "adjoint_film":
        g.set_hext_field(torch.zeros(3 * f.ncells, device="cuda:0"))
    md = torch.from_numpy(m0.reshape(-1)).cuda()
    g.set_m(md)
    if name == "adjoint_film":
        tape = g.step_checkpointed(steps, w.dt, 16)
        lam = torch.full((3 * f.ncells,), 1e-6, device="cuda:0")
        gh = torch.zeros(3 * f.ncells, device="cuda:0")
        gm = torch.zeros(f.ncells, device="cuda:0")
        g.backward(lam, steps, w.dt, 16, gh, gm, tape=tape)
    else:
        g.step(steps, w.dt)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": name, "steps": steps}), flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank (replicas: weak scaling)."""
    return units_per_rank * world * steps / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    csrc = os.path.join(ROOT, "paper_1411_2565_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernels are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("kernels", {}).get(workload, {}).get(kernel)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.rows = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for n, v in zip(names, r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def algorithmic_bytes(g, film):
    """Compulsory bytes of one launch of each kernel (each operand read once, result written
    once).  Films with nz <= 4 take the fused path (x pass, fused y pass with the direct z
    sum); thicker ones the split path (x pass, y FFT launched forward and inverse, z pass)."""
    nx, ny, nz = film.grid
    Px = 1
    while Px < 2 * nx - 1:
        Px *= 2
    Py = 1
    while Py < 2 * ny - 1:
        Py *= 2
    Kx, Ky = Px // 2 + 1, Py // 2 + 1
    N = nx * ny * nz
    spec = 3 * nz * Kx * ny * 8                    # x-transformed rows: [3][nz][Kx][ny] complex
    x_fast = 2 * spec + 2 * 12 * N                 # read S and m, write S and m
    if nz <= 4:
        nslot = 4 if nz == 1 else 6 * nz - 2
        tensor = Kx * nslot * Ky * 4
        return {"yz_fast": 2 * spec + tensor,      # read S and T, write S
                "x_fast": x_fast,
                "per_cell": (4 * spec + tensor + 24 * N) / N}
    Pz = 1
    while Pz < 2 * nz - 1:
        Pz *= 2
    A1, A2 = Kx * ny * nz, Kx * Py * nz
    tensor = Kx * Ky * (Pz // 2 + 1) * 6 * 4
    y_fast = 24 * A1 + 24 * A2                     # either direction: ny rows <-> Py rows
    z_fast = 48 * A2 + tensor                      # read and write the Py rows, read T
    return {"x_fast": x_fast, "y_fast": y_fast, "z_fast": z_fast,
            "per_cell": (x_fast + 2 * y_fast + z_fast) / N}


def kernel_rooflines(trace, byt, peak, peak_kind, workload):
    """Per traced kernel: average launch time, algorithmic bytes per launch, achieved GB/s
    and its fraction of the HBM peak, and the profiled DRAM bytes per launch (or None)."""
    out = {}
    for k, (ms, n) in trace.items():
        if k not in byt:
            continue
        avg = ms / n * 1e-3
        gbs = byt[k] / avg / 1e9
        out[k] = {"launches": n, "avg_launch_us": round(avg * 1e6, 2), "bytes_per_launch": byt[k],
                  "achieved": round(gbs, 1), "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                  "frac": round(gbs / peak, 4), "traffic": recorded_traffic(k, workload)}
    return out


def five_pass_bytes(film):
    """Bytes per step of a design that keeps every intermediate spectrum in HBM: x R2C
    (12N in, 24 A1 out), y FFT (24 A1 in, 24 A2 out), z FFT + product + inverse z (24 A2 in,
    T, 24 A2 out), inverse y (24 A2 in, 24 A1 out), x C2R + step (24 A1 + 12N in, 12N out);
    for nz = 1 the y pass takes the product (T) and there is no z pass.  A1 = Kx ny nz and
    A2 = Kx Py nz complex points, T the tensor octant (6 or 4 components)."""
    nx, ny, nz = film.grid
    def pad(n):
        p = 1
        while p < 2 * n - 1:
            p *= 2
        return p
    Px, Py, Pz = pad(nx), pad(ny), pad(nz)
    Kx, Ky, Kz = Px // 2 + 1, Py // 2 + 1, Pz // 2 + 1
    N = nx * ny * nz
    A1, A2 = Kx * ny * nz, Kx * Py * nz
    if nz == 1:
        T = Kx * Ky * 4 * 4
        return 12 * N + 24 * A1 + 24 * A1 + T + 24 * A1 + 24 * A1 + 12 * N + 12 * N
    T = Kx * Ky * Kz * 6 * 4
    return (12 * N + 24 * A1 + 24 * A1 + 24 * A2 + 24 * A2 + T + 24 * A2 + 24 * A2 + 24 * A1 + 24 * A1
            + 12 * N + 12 * N)


def run_grace(args, rank, world, local):
    import numpy as np
    import torch

    import workloads
    from paper_1411_2565_gb300 import _lib
    from paper_1411_2565_gb300 import build as libbuild
    from paper_1411_2565_gb300.grace import Grace

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    libbuild.build()
    w = getattr(workloads, args.workload)()
    f, m0 = w.films[0], w.m0[0]
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=dev)   # tuned schedule
    options = g.options
    g.set_hext(f.hext)
    m_dev = torch.from_numpy(m0.reshape(-1)).to(dev)
    g.set_m(m_dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        flush.zero_()
        g.step(1, w.dt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a, b in ev:
        flush.zero_()
        a.record(s)
        g.step(1, w.dt)
        b.record(s)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ncell = f.ncells
    value = whole_job_rate(ncell, world, args.steps, total_ms * 1e-3)
    # the timed loop in five equal chunks: their rates' median, min and max
    chunk = max(1, args.steps // 5)
    rates = sorted(ncell * chunk / (sum(step_ms[i * chunk:(i + 1) * chunk]) * 1e-3) for i in range(5)
                   if len(step_ms) >= (i + 1) * chunk)
    runs = {"chunks": len(rates), "steps_per_chunk": chunk, "median": rates[len(rates) // 2],
            "min": rates[0], "max": rates[-1]} if rates else None

    # per-kernel durations: the same flushed single steps again, with an event pair around
    # every kernel (the events separate the kernels, so this pass is not the headline)
    ktr = min(args.steps, 1000)
    g.trace(2 * ktr + 8)
    for _ in range(ktr):
        flush.zero_()
        g.step(1, w.dt)
    trace = g.trace_read()
    g.trace(0)

    # dominant kernel and its roofline
    peak, peak_kind = measured_peaks()
    byt = algorithmic_bytes(g, f)
    # the whole step against the HBM peak: `frac_moved` takes the bytes this design moves
    # (every kernel's arrays read and written once) and is the step's roofline fraction;
    # `frac_five_pass_model` (every intermediate spectrum through HBM, bytes this design
    # does not move) is only a labelled comparison
    step_s = total_ms * 1e-3 / args.steps
    moved_b = byt["per_cell"] * ncell
    model_b = five_pass_bytes(f)
    step_roof = {"unit": "GB/s", "peak": peak, "peak_source": peak_kind, "step_us": round(step_s * 1e6, 2),
                 "bytes_moved": int(moved_b), "frac_moved": round(moved_b / step_s / 1e9 / peak, 4),
                 "bytes_five_pass_model": int(model_b),
                 "frac_five_pass_model": round(model_b / step_s / 1e9 / peak, 4)}
    dom = max(trace.items(), key=lambda kv: kv[1][0])[0] if trace else None
    roof = None
    if dom in byt:
        avg_ms = trace[dom][0] / trace[dom][1]
        achieved = byt[dom] / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "bytes_per_launch": byt[dom], "avg_launch_us": round(avg_ms * 1e3, 2),
                "traffic": recorded_traffic(dom, args.workload),
                "timing": f"CUDA events around each kernel over {ktr} flushed steps"}
    kernels = {k: {"avg_us": round(v[0] / v[1] * 1e3, 2), "launches": v[1],
                   "share": round(v[0] / sum(x[0] for x in trace.values()), 3)}
               for k, v in trace.items()}

    # end to end through the C ABI with host buffers: every step copies its input m from
    # page-locked host memory (grace_set_m_host), takes one step and copies the result back
    # (grace_get_m_host_async).  The steps are independent, so E2E_HANDLES handles on as many
    # streams take the steps in turn: one's copies and kernels overlap the others'; a handle
    # waits for its previous result before it starts its next step.
    g.close()
    streams = [torch.cuda.Stream(device=dev) for _ in range(E2E_HANDLES)]
    ctxs = [Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=dev, stream=st) for st in streams]
    for c in ctxs:
        c.set_hext(f.hext)
    host_in = [torch.from_numpy(m0.reshape(-1).copy()).pin_memory() for _ in range(E2E_HANDLES)]
    host_out = [torch.empty_like(host_in[0]).pin_memory() for _ in range(E2E_HANDLES)]
    for k in range(E2E_HANDLES):           # untimed: one pass through each handle
        ctxs[k].set_m_host(host_in[k].numpy())
        ctxs[k].step(1, w.dt)
        ctxs[k].get_m_host(host_out[k].numpy(), wait=False)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        i = k % E2E_HANDLES
        streams[i].synchronize()           # the handle's previous result has arrived
        ctxs[i].set_m_host(host_in[i].numpy())
        ctxs[i].step(1, w.dt)
        ctxs[i].get_m_host(host_out[i].numpy(), wait=False)
    for st in streams:
        st.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": whole_job_rate(ncell, world, args.e2e_steps, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 12 * ncell, "d2h_bytes_per_step": 12 * ncell,
           "steps": args.e2e_steps, "handles": E2E_HANDLES,
           "path": "grace_set_m_host + grace_step(1) + grace_get_m_host_async per step, handles on "
                   "separate streams taking the steps in turn (host wall clock, all copies inside)"}
    e2e["results_identical_across_handles"] = bool(all(torch.equal(host_out[0], o) for o in host_out[1:]))
    for c in ctxs:
        c.close()

    extras = None
    if rank == 0 and not args.no_extras:
        extras = extra_workloads(dev, args.workload)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)
        if args.cpu_procs != 0:
            cpu["all_cores"] = cpu_baseline_all_cores(args.workload, args.cpu_seconds, args.cpu_procs)
    launches = sum(v[1] for v in trace.values()) // max(1, ktr) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "cells": ncell, "cell_m": list(f.cell), "dt_s": w.dt,
                   "padded": [int(2 ** math.ceil(math.log2(max(1, 2 * n - 1)))) for n in f.grid],
                   "initial_state": w.note, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}", "wall_s_timed_loop": round(wall, 3),
                   "options": {_lib.OPT_NAMES[k]: v for k, v in sorted(options.items())},
                   "options_source": "autotuned schedule (local cache, else the shipped GB300 table)"
                                     if options else "library defaults (no tuned schedule for this shape)"},
        "roofline": roof, "step_roofline": step_roof, "runs_of_5": runs,
        "kernels": kernels, "gpu_launches": launches, "e2e": e2e,
        "cpu_baseline": cpu, "clocks": clk, "workloads": extras,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_events(fn, reps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3


def plain_workload_extra(dev, name, flush, steps=200):
    """Another plain single-film workload beside the headline: `steps` single steps with L2
    flushed before each, the per-kernel split from traced steps, per-kernel rooflines and
    the whole step against the HBM peak."""
    import torch

    import workloads
    from paper_1411_2565_gb300.grace import Grace
    w = getattr(workloads, name)()
    f, m0 = w.films[0], w.m0[0]
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=dev)
    g.set_hext(f.hext)
    g.set_m(torch.from_numpy(m0.reshape(-1)).to(dev))
    g.step(5, w.dt)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        g.step(1, w.dt)
        b.record()
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    g.trace(8 * steps)
    for _ in range(steps):
        flush.zero_()
        g.step(1, w.dt)
    tr = g.trace_read()
    g.trace(0)
    g.close()
    from paper_1411_2565_gb300 import _lib
    opts = {_lib.OPT_NAMES[k]: v for k, v in sorted(g.options.items())}
    peak, peak_kind = measured_peaks()
    byt = algorithmic_bytes(g, f)
    step_s = t / steps
    moved = byt["per_cell"] * f.ncells
    return {"workload": w.name, "value": f.ncells * steps / t, "unit": UNIT,
            "ms_per_step": step_s * 1e3, "options": opts,
            "kernels_us": {k: round(v[0] / v[1] * 1e3, 1) for k, v in tr.items()},
            "roofline": kernel_rooflines(tr, byt, peak, peak_kind, name),
            "step_roofline": {
                "unit": "GB/s", "peak": peak, "peak_source": peak_kind, "bytes_moved": int(moved),
                "frac_moved": round(moved / step_s / 1e9 / peak, 4),
                "bytes_five_pass_model": int(five_pass_bytes(f)),
                "frac_five_pass_model": round(five_pass_bytes(f) / step_s / 1e9 / peak, 4)},
            "method": f"{steps} single steps, L2 flushed before each; kernel times from "
                      f"{steps} more traced steps"}


def extra_workloads(dev, headline):
    """Throughput of the other forms of the hot path: the other plain workload (film or
    block), the film ensemble, the adjoint, the cube sweep and a vendor-FFT comparison."""
    import numpy as np
    import torch

    import workloads
    from paper_1411_2565_gb300.grace import Grace, GraceBatch
    out = {}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peak, peak_kind = measured_peaks()
    for name in ("block", "film_large"):
        if name != headline:
            out[name] = plain_workload_extra(dev, name, flush)
    # 256-film ensemble, 2000 steps in replayed CUDA graphs: the tuned schedule, and both
    # batch paths explicitly (grouped launches per size class on side streams; one
    # persistent cooperative launch per graph)
    from paper_1411_2565_gb300 import _lib
    w = workloads.ensemble()
    m_all = torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).to(dev)
    ncell = sum(f.ncells for f in w.films)
    paths = {}
    for name, opts in (("grouped", {_lib.OPT_PERSISTENT: 0}), ("persistent", {_lib.OPT_PERSISTENT: 1})):
        gb = GraceBatch(w.films, device=dev, options=opts)
        gb.set_m(m_all)
        gb.step(32, w.dt)
        tp = time_events(lambda: gb.step(2000, w.dt), 1)
        gb.sync()
        paths[name] = {"value": ncell * 2000 / tp, "ms_per_step": tp / 2000 * 1e3}
        gb.close()
    gb = GraceBatch(w.films, device=dev)
    gb.set_m(m_all)
    gb.step(32, w.dt)
    t = time_events(lambda: gb.step(2000, w.dt), 1)
    fused_b = sum(algorithmic_bytes(None, fi)["per_cell"] * fi.ncells for fi in w.films)
    model_b = sum(five_pass_bytes(fi) for fi in w.films)
    step_s = t / 2000
    out["ensemble"] = {"workload": w.name, "films": len(w.films), "cells": ncell,
                       "options": {_lib.OPT_NAMES[k]: v for k, v in sorted(gb.options.items())},
                       "paths": paths,
                       "value": ncell * 2000 / t, "unit": UNIT, "ms_per_step": t / 2000 * 1e3,
                       "step_roofline": {
                           "unit": "GB/s", "peak": peak, "peak_source": peak_kind,
                           "bytes_moved": int(fused_b), "frac_moved": round(fused_b / step_s / 1e9 / peak, 4),
                           "bytes_five_pass_model": int(model_b),
                           "frac_five_pass_model": round(model_b / step_s / 1e9 / peak, 4)},
                       "method": "2000 steps back to back (graphs of 16 steps); ~300 MB working set"}
    del gb
    # adjoint film at its stated length: 4,096 forward steps, then the backward pass
    # (checkpoints every 64): the forward that keeps its checkpoints and the adjoint from
    # them (the autograd path), and the self-contained grace_backward, which collects the
    # checkpoints in a forward pass of its own
    w = workloads.adjoint_film()
    f, m0 = w.films[0], w.m0[0]
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=dev)
    ms = torch.from_numpy(w.ms_field.reshape(-1)).to(dev)
    h = torch.zeros(3 * f.ncells, device=dev)
    g.set_ms_field(ms)
    g.set_hext_field(h)
    md = torch.from_numpy(m0.reshape(-1)).to(dev)
    n = w.steps
    g.set_m(md)
    g.step(n, w.dt)                              # warm-up (graph capture)
    g.set_m(md)
    t_f = time_events(lambda: g.step(n, w.dt), 1)
    lam = torch.full((3 * f.ncells,), 1e-6, device=dev)
    gh = torch.zeros_like(h)
    gm = torch.zeros_like(ms)
    g.set_m(md)
    tape = g.step_checkpointed(n, w.dt, 64)      # warm-up (scratch allocation by torch)
    g.backward(lam, n, w.dt, 64, gh, gm, tape=tape)
    del tape                                     # its block returns to torch's cache for the next tape
    g.set_m(md)
    tapes = []
    t_fc = time_events(lambda: tapes.append(g.step_checkpointed(n, w.dt, 64)), 1)
    t_bc = time_events(lambda: g.backward(lam, n, w.dt, 64, gh, gm, tape=tapes[-1]), 1)
    g.backward(lam, n, w.dt, 64, gh, gm)         # warm-up
    t_b = time_events(lambda: g.backward(lam, n, w.dt, 64, gh, gm), 1)
    out["adjoint"] = {"workload": w.name, "steps": n, "unit": UNIT,
                      "forward_value": f.ncells * n / t_f,
                      "forward_checkpointed_value": f.ncells * n / t_fc,
                      "backward_value": f.ncells * n / t_bc,
                      "backward_over_forward": t_bc / t_f,
                      "fwd_plus_bwd_ms_per_step": (t_fc + t_bc) / n * 1e3,
                      "self_contained_backward_value": f.ncells * n / t_b,
                      "self_contained_backward_over_forward": t_b / t_f,
                      "method": "grace_step (forward), grace_step_checkpointed then "
                                "grace_backward_checkpointed (backward: re-computes each segment "
                                "from its checkpoint), checkpoints every 64; self-contained: "
                                "grace_backward with its own checkpointing forward pass"}
    del g
    out["cufft_demag_comparison"] = {name: cufft_demag_comparison(dev, flush, name)
                                     for name in ("block", "film_large")}
    out["cube_sweep"] = cube_sweep(dev)
    return out


# the paper's Table 1: per-step time of its GPU code (HD 7970) for N^3 cubes, context only
PAPER_TABLE1_GPU_MS = {8: 1.95, 16: 2.723, 32: 3.151, 64: 6.558, 128: 26.34}


def cube_sweep(dev, steps=64):
    """N^3 cubes of 1 nm cells in the paper's Table 1 material (A = 1e-11 J/m, Ms = 1e6 A/m,
    H_anis = 100 kA/m along x, so Ku = mu0 Ms H_anis / 2), random unit m, dt = 1e-14 s:
    cell-steps/s in graphs of 16 steps (working sets up to ~0.4 GB, L2 not flushed), next
    to the paper's own per-step times (other hardware, context only)."""
    import math
    import torch

    import workloads
    from paper_1411_2565_gb300.grace import Grace
    Ms, A, HK = 1e6, 1e-11, 1e5
    Ku = 4e-7 * math.pi * Ms * HK / 2
    res = {}
    for n in sorted(PAPER_TABLE1_GPU_MS):
        g = Grace((n, n, n), (1e-9, 1e-9, 1e-9), Ms, A, Ku, 0.1, device=dev)
        g.set_m(torch.from_numpy(workloads.random_unit_m((n, n, n), seed=40 + n).reshape(-1)).to(dev))
        g.step(32, 1e-14)
        t = time_events(lambda: g.step(steps, 1e-14), 1)
        g.close()
        ms = t / steps * 1e3
        res[f"{n}^3"] = {"cells": n ** 3, "ms_per_step": round(ms, 4), "value": n ** 3 / (ms * 1e-3),
                         "paper_gpu_ms_per_step": PAPER_TABLE1_GPU_MS[n],
                         "ratio_to_paper": round(PAPER_TABLE1_GPU_MS[n] / ms, 1)}
    return res


def cufft_demag_comparison(dev, flush, name="film_large", reps=20):
    """Timed comparison only (not the product path): a workload's demag convolution done
    with the vendor FFT through torch.fft on the same zero-padded grid, FP32: R2C of the
    three padded components, the 6-component symmetric tensor product, C2R and crop.
    The tensor values are placeholders of the right shape (timing does not depend on them)."""
    import torch

    import workloads
    w = getattr(workloads, name)()
    f = w.films[0]
    nx, ny, nz = f.grid
    Px, Py, Pz = (1 << (2 * n - 1 - 1).bit_length() if n > 1 else 1 for n in (nx, ny, nz))
    m = torch.zeros(3, Pz, Py, Px, device=dev)
    m[:, :nz, :ny, :nx] = torch.randn(3, nz, ny, nx, device=dev)
    T = torch.randn(6, Pz, Py, Px // 2 + 1, device=dev)

    def conv():
        X = torch.fft.rfftn(m, dim=(1, 2, 3))
        H = torch.stack([T[0] * X[0] + T[3] * X[1] + T[4] * X[2],
                         T[3] * X[0] + T[1] * X[1] + T[5] * X[2],
                         T[4] * X[0] + T[5] * X[1] + T[2] * X[2]])
        h = torch.fft.irfftn(H, s=(Pz, Py, Px), dim=(1, 2, 3))
        return h[:, :nz, :ny, :nx].contiguous()

    conv()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        conv()
        b.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / reps
    return {"workload": w.name, "padded": [Px, Py, Pz], "ms_per_demag": round(ms, 4),
            "equivalent_cell_steps_per_s": f.ncells / (ms * 1e-3),
            "method": "torch.fft.rfftn / irfftn (vendor FFT) + elementwise tensor product, FP32, "
                      f"L2 flushed before each of {reps} evaluations; demag only, no exchange or step"}


def cpu_baseline(w, seconds):
    """The FP64 oracle as it stands, on the host cores, for a bounded number of steps."""
    import numpy as np

    from oracle import llg
    f, m0 = w.films[0], w.m0[0]
    p = llg.Params(f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, f.hext)
    nx, ny, nz = f.grid
    D = llg.Demag((nx, ny, nz), f.cell)          # tensor spectrum: set-up, not timed
    m = m0.astype(np.float64)
    t0 = time.perf_counter()
    n = 0
    while True:
        m = llg.euler_step(m, p, w.dt, D)
        n += 1
        if time.perf_counter() - t0 >= seconds or n >= 1000:
            break
    dt = time.perf_counter() - t0
    return {"value": f.ncells * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 Euler steps of the full {w.name} film (numpy FFT convolution, "
                      f"single thread), {dt:.1f} s", "steps": n, "seconds": dt}


def _oracle_replica(name, seconds, barrier, results):
    """One oracle replica (a spawned process): its own film and tensor spectrum, then Euler
    steps for `seconds` once every replica is ready."""
    import numpy as np

    import workloads
    from oracle import llg
    w = getattr(workloads, name)()
    f, m0 = w.films[0], w.m0[0]
    p = llg.Params(f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, f.hext)
    D = llg.Demag(f.grid, f.cell)
    m = m0.astype(np.float64)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    n = 0
    while True:
        m = llg.euler_step(m, p, w.dt, D)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    results.put((n, time.perf_counter() - t0, f.ncells))


# host memory one oracle replica holds (FP64 state, padded FFT buffers, tensor spectrum), bytes
ORACLE_REPLICA_BYTES = {"block": 7 << 30, "film_large": 2 << 30, "film_small": 1 << 30}


def cpu_baseline_all_cores(name, seconds, procs=-1):
    """The same oracle on every host core: independent replicas of the workload in spawned
    processes (the oracle itself is single-threaded), timed over a common window.  The
    replica count is capped by the host memory (ORACLE_REPLICA_BYTES per replica: about
    7 GB for the block, 2 GB for film_large)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = cores if procs < 0 else min(procs, cores)
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        n = max(1, min(n, int(avail // ORACLE_REPLICA_BYTES.get(name, 2 << 30))))
    except (ValueError, OSError, AttributeError):
        pass
    ctx = mp.get_context("spawn")             # never fork a process that holds a CUDA context
    barrier, results = ctx.Barrier(n), ctx.Queue()
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ.update({k: "1" for k in env})
    import queue
    ps, out = [], []
    try:
        ps = [ctx.Process(target=_oracle_replica, args=(name, seconds, barrier, results)) for _ in range(n)]
        for p in ps:
            p.start()
        deadline = time.time() + 900
        while len(out) < n:
            try:
                out.append(results.get(timeout=2))
            except queue.Empty:
                if time.time() > deadline or any(p.exitcode not in (None, 0) for p in ps):
                    return {"unavailable": "an oracle replica failed or did not finish", "cores": n}
        for p in ps:
            p.join()
    finally:
        for p in ps:                          # only the replicas started here
            if p.is_alive():
                p.terminate()
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    steps = sum(o[0] for o in out)
    value = sum(o[0] * o[2] / o[1] for o in out)
    return {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "replicas": n,
            "sample": f"{n} single-threaded oracle replicas of the full {name} film, one per core, "
                      f"{steps} FP64 Euler steps in all over ~{seconds:.0f} s",
            "steps": steps, "seconds": max(o[1] for o in out)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import workloads
    w = getattr(workloads, args.workload)()
    budget = max(5.0, min(150.0, args.cpu_seconds * 3))
    f = w.films[0]
    cb = None
    if args.cpu_procs != 1:
        # every host core: independent single-threaded replicas of the oracle
        cb = cpu_baseline_all_cores(args.workload, budget, args.cpu_procs)
        if "unavailable" in cb:
            cb = None
    if cb is None:
        cb = cpu_baseline(w, budget)
    line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": cb["steps"], "warmup": 0, "ms_per_step": f.ncells / cb["value"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "cells": f.ncells, "dt_s": w.dt,
                       "note": "reference arm = the FP64 CPU oracle on the host cores (one "
                               "single-threaded replica per core); each timed step is one oracle "
                               "Euler step of the full film, as many as fit the time budget; "
                               "ms_per_step = cells / aggregate rate"},
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "requested": {"steps": args.steps, "warmup": args.warmup,
                          "note": "the oracle runs as many full-film steps as fit its time budget"},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_run:
        profile_run(args.profile_run, args.steps)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_grace(args, rank, world, local)


if __name__ == "__main__":
    main()
