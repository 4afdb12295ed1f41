"""Autotuner for the launch schedule of a film or an ensemble.

For a given set of films it times each candidate schedule on the real device with CUDA
events and keeps the fastest.  The candidates are the FFT tiles and schedules (x-pass lines per
block: one line or the larger compiled tile; kx columns per fused y block; the z pass at 16
points per thread where the padded z length is 128, or 256- or 128-thread blocks at 8
points per thread), the batch grouping (the
launch groups of an ensemble stepping side by side on streams of their own, one after
another, or all in one persistent cooperative launch) and the steps per captured CUDA graph.
A single film is timed the way the benchmark steps it — single steps, L2 flushed before
each — and a batch by warm replays of captured graphs, the way an ensemble is stepped.
Options that cannot affect the timing (a z tile for films without an FFT along z, side
streams and the graph length for one film) keep their defaults instead of multiplying
the search; programmatic dependent launch stays on (captured graphs do not use it, and
for single-step calls it measured faster).

Results are cached in a JSON file keyed by the film shapes and the device name.
``Grace`` and ``GraceBatch`` apply ``best()`` by default — the local cache, else the table
shipped with the package (``tuned_gb300.json``, written by ``python -m
paper_1411_2565_gb300.autotune``), else the library's own heuristics.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
from typing import Dict, List, Sequence

import numpy as np
import torch

from . import _lib

CACHE = os.environ.get("GRACE_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "grace_gb300_autotune.json"))
# schedules tuned on a GB300 for the benchmark shapes, shipped with the package
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")

CANDIDATES = {
    _lib.OPT_TILE_X: (0, 1, 2),
    _lib.OPT_TILE_YZ: (0, 1, 2, 4),
    _lib.OPT_TILE_Z: (0, 1, 2, 4),
    _lib.OPT_SIDE_STREAMS: (1, 0),
    _lib.OPT_PERSISTENT: (0, 1),
    _lib.OPT_GRAPH_STEPS: (8, 16, 32),
    _lib.OPT_PDL: (0, 1),
}
DEFAULTS = {_lib.OPT_TILE_X: 0, _lib.OPT_TILE_YZ: 0, _lib.OPT_TILE_Z: 0, _lib.OPT_SIDE_STREAMS: 1,
            _lib.OPT_PERSISTENT: 0, _lib.OPT_GRAPH_STEPS: 16, _lib.OPT_PDL: 1}
BIND_OPTIONS = (_lib.OPT_TILE_X, _lib.OPT_TILE_YZ, _lib.OPT_TILE_Z, _lib.OPT_PERSISTENT)


def relevant(films) -> Dict[int, bool]:
    """Which options can change how these films run (the rest keep DEFAULTS)."""
    thin = any(f.grid[2] <= 4 for f in films)
    thick = any(f.grid[2] > 4 for f in films)
    batch = len(films) > 1
    return {_lib.OPT_TILE_X: True, _lib.OPT_TILE_YZ: thin, _lib.OPT_TILE_Z: thick,
            _lib.OPT_SIDE_STREAMS: batch, _lib.OPT_PERSISTENT: batch and thin and not thick,
            _lib.OPT_GRAPH_STEPS: batch, _lib.OPT_PDL: False}


def _key(films, device) -> str:
    shapes = sorted(f"{f.grid}|{f.cell}" for f in films)
    name = torch.cuda.get_device_name(device)
    return hashlib.sha256(("|".join(shapes) + "|" + name).encode()).hexdigest()[:24]


def _load() -> Dict:
    if os.path.exists(CACHE):
        with open(CACHE) as fh:
            return json.load(fh)
    return {}


def _store(d: Dict):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1)
    os.replace(tmp, CACHE)


L2_FLUSH_BYTES = 256 << 20   # more than the GB300's 129 MB L2


def _time(films, m0s, dt, options, device, steps=64, reps=3) -> float:
    """ms per step of these films under `options`.  One film: single steps with L2 flushed
    before each (a large film's step in production finds little of its data in L2, and a
    small film's launch latency shows); a batch: warm replays of captured graphs (how an
    ensemble is stepped)."""
    from .grace import Grace, GraceBatch
    bind = {k: v for k, v in options.items() if k in BIND_OPTIONS}
    if len(films) == 1:
        f = films[0]
        g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=device, options=bind)
        g.set_hext(f.hext)
    else:
        g = GraceBatch(films, device=device, options=bind)
    for k, v in options.items():
        if k not in BIND_OPTIONS:
            g.set_option(k, v)
    g.set_m(torch.from_numpy(np.concatenate([m.reshape(-1) for m in m0s])).to(device))
    g.step(steps, dt)
    if len(films) == 1:
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record()
            g.step(1, dt)
            b.record()
        torch.cuda.synchronize()
        g.close()
        return float(np.median([a.elapsed_time(b) for a, b in ev]))
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.step(steps, dt)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / steps)
    g.close()
    return best


def tune(films: Sequence, m0s: Sequence[np.ndarray], dt: float, device="cuda", force=False) -> Dict[int, int]:
    """Time every candidate schedule for these films; returns and caches the best options."""
    device = torch.device(device)
    cache = _load()
    key = _key(films, device)
    if key in cache and not force:
        return {int(k): v for k, v in cache[key]["options"].items()}
    results = []
    use = relevant(films)
    names = list(CANDIDATES)
    for values in itertools.product(*(CANDIDATES[n] if use[n] else (DEFAULTS[n],) for n in names)):
        opts = dict(zip(names, values))
        try:
            ms = _time(films, m0s, dt, opts, device)
        except _lib.GraceError:
            continue                       # a tile this shape does not support
        results.append((ms, opts))
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    cache[key] = {"options": {str(k): v for k, v in best.items()}, "ms_per_step": best_ms,
                  "films": len(films), "tried": len(results)}
    _store(cache)
    return best


def best(films: Sequence, device="cuda") -> Dict[int, int]:
    """Cached options for these films: the local cache, else the shipped GB300 table, else {}.
    An entry that predates an option gets that option's default."""
    key = _key(films, torch.device(device))
    entry = _load().get(key)
    if entry is None and os.path.exists(SHIPPED):
        with open(SHIPPED) as fh:
            entry = json.load(fh).get(key)
    if entry is None:
        return {}
    opts = dict(DEFAULTS)
    opts.update({int(k): v for k, v in entry["options"].items()})
    return opts


def main(argv=None):
    """Tune the benchmark workloads on this device and write the table ``best`` ships with."""
    import argparse
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--workloads", default="block,film_large,film_small,ensemble,adjoint_film")
    ap.add_argument("--out", default=SHIPPED)
    args = ap.parse_args(argv)
    table = {}
    if os.path.exists(args.out):
        with open(args.out) as fh:
            table = json.load(fh)
    for name in args.workloads.split(","):
        w = getattr(workloads, name)()
        opts = tune(w.films, w.m0, w.dt, force=True)
        key = _key(w.films, torch.device("cuda"))
        entry = _load()[key]
        entry["workload"] = w.name
        table[key] = entry
        print(name, {k: v for k, v in opts.items()}, f"{entry['ms_per_step']:.4f} ms/step", flush=True)
    tmp = args.out + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1)
    os.replace(tmp, args.out)


if __name__ == "__main__":
    main()
