"""Standard-problem-4-shaped reversal run (Sec. 4): a 500 x 125 x 3 nm permalloy-like film
(A = 1.3e-11 J/m, Ms = 8.0e5 A/m, no anisotropy) is relaxed at large damping from a
near-saturated state along [1,1,1] into the S-state, then reversed at alpha = 0.02 by
field 1 (-24.6, 4.3, 0) mT or field 2 (-35.5, -6.3, 0) mT.

The paper discretises the film in 1 nm cells; here the discretisation is a parameter
(cells of 500/nx x 125/ny x 3 nm, one layer), with the time step scaled by the square of
the in-plane cell size so that the explicit step sees the same exchange stiffness.  The
applied field of the reversal is switched on at t = 0 through the same start / decay /
stop envelope as the paper's input file (on from 0, decay starting after the run).

Runs entirely on the GPU through the C ABI; <m> is sampled with grace_energy.

    python -m paper_1411_2565_gb300.mumag4 --grid 128x32 --field 1
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

MU0 = 4e-7 * math.pi
FILM_NM = (500.0, 125.0, 3.0)
A_EX, MS = 1.3e-11, 8.0e5
FIELDS_MT = {1: (-24.6, 4.3, 0.0), 2: (-35.5, -6.3, 0.0)}
DT_COARSE = 1e-14          # s, for 500/128 nm cells; scaled by (cell / that)^2


@dataclass
class Run:
    grid: Sequence[int]
    field: int
    dt: float
    relax_m: List[float]
    t: List[float] = field(default_factory=list)         # s, from the field switch-on
    mavg: List[List[float]] = field(default_factory=list)
    t_cross: Optional[float] = None                     # first zero of <m_x> (interpolated)
    m_cross: Optional[np.ndarray] = None                # state at the first sample past it
    m_relaxed: Optional[np.ndarray] = None
    m_final: Optional[np.ndarray] = None
    wall_s: float = 0.0
    steps: int = 0


def cell_size(grid) -> tuple:
    nx, ny = grid[0], grid[1]
    return (FILM_NM[0] * 1e-9 / nx, FILM_NM[1] * 1e-9 / ny, FILM_NM[2] * 1e-9)


def time_step(grid) -> float:
    c = cell_size(grid)[0]
    return DT_COARSE * (c / (FILM_NM[0] * 1e-9 / 128)) ** 2


def field_Apm(k: int) -> tuple:
    return tuple(b * 1e-3 / MU0 for b in FIELDS_MT[k])


def _grace(grid, alpha, device, integrator):
    from .grace import Grace
    from . import _lib
    opts = {_lib.OPT_INTEGRATOR: 1} if integrator == "heun" else None
    return Grace((grid[0], grid[1], 1), cell_size(grid), MS, A_EX, 0.0, alpha, device=device,
                 options=opts)


def relax(grid, m0: np.ndarray, t_relax: float = 2e-9, alpha: float = 0.5, device="cuda:0",
          integrator="euler"):
    """Relax m0 ([3][1][ny][nx], e.g. near-saturated along [1,1,1]) in zero field for t_relax;
    returns the state."""
    import torch
    g = _grace(grid, alpha, device, integrator)
    m = m0
    g.set_m(torch.from_numpy(m.reshape(-1)).to(device))
    dt = time_step(grid)
    g.step(int(round(t_relax / dt)), dt)
    out = g.get_m().cpu().numpy().reshape(m.shape)
    g.close()
    return out


def reverse(grid, m_relaxed: np.ndarray, field_no: int = 1, t_run: float = 1e-9, sample: float = 1e-12,
            alpha: float = 0.02, device="cuda:0", integrator="euler") -> Run:
    """Apply field `field_no` at t = 0 to the relaxed state and sample <m> every `sample` s."""
    import torch
    g = _grace(grid, alpha, device, integrator)
    g.set_hext(field_Apm(field_no))
    g.set_hext_pulse((0.0, t_run, 2.0 * t_run))   # on from 0, constant for the run
    g.time = 0.0
    g.set_m(torch.from_numpy(m_relaxed.reshape(-1)).to(device))
    dt = time_step(grid)
    per = max(1, int(round(sample / dt)))
    nsamp = int(round(t_run / (per * dt)))
    _, m_start = g.energy()
    r = Run(grid=tuple(grid), field=field_no, dt=dt, relax_m=list(map(float, m_start)),
            m_relaxed=m_relaxed)
    r.t.append(0.0)
    r.mavg.append(list(map(float, m_start)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nsamp):
        g.step(per, dt)
        _, mv = g.energy()
        r.t.append(g.time)
        r.mavg.append(list(map(float, mv)))
        if r.t_cross is None and r.mavg[-2][0] > 0.0 >= mv[0]:
            a, b = r.mavg[-2][0], mv[0]
            r.t_cross = r.t[-2] + (r.t[-1] - r.t[-2]) * a / (a - b)
            r.m_cross = g.get_m().cpu().numpy().reshape(m_relaxed.shape)
    r.wall_s = time.perf_counter() - t0
    r.steps = nsamp * per
    r.m_final = g.get_m().cpu().numpy().reshape(m_relaxed.shape)
    g.close()
    return r


def curve_distance(a: Run, b: Run) -> float:
    """max over common sample times and components of |<m>_a - <m>_b| (sampled on the same
    times by linear interpolation of b)."""
    ta, tb = np.asarray(a.t), np.asarray(b.t)
    ma, mb = np.asarray(a.mavg), np.asarray(b.mavg)
    d = 0.0
    for c in range(3):
        d = max(d, float(np.abs(ma[:, c] - np.interp(ta, tb, mb[:, c])).max()))
    return d


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--grid", default="128x32", help="in-plane cells nx x ny over 500 x 125 nm")
    ap.add_argument("--field", type=int, default=1, choices=(1, 2))
    ap.add_argument("--relax-ns", type=float, default=2.0)
    ap.add_argument("--run-ns", type=float, default=1.0)
    ap.add_argument("--sample-ps", type=float, default=10.0)
    ap.add_argument("--integrator", default="euler", choices=("euler", "heun"))
    args = ap.parse_args(argv)
    grid = tuple(int(v) for v in args.grid.lower().split("x"))
    import workloads                      # seeded input generators (repository root)
    m0 = workloads.near_saturated_m((1, grid[1], grid[0]), (1.0, 1.0, 1.0), seed=10)
    mr = relax(grid, m0, args.relax_ns * 1e-9, integrator=args.integrator)
    r = reverse(grid, mr, args.field, args.run_ns * 1e-9, args.sample_ps * 1e-12, integrator=args.integrator)
    print(json.dumps({"grid": grid, "field": args.field, "dt_s": r.dt, "relaxed_m": r.relax_m,
                      "t_cross_ns": None if r.t_cross is None else r.t_cross * 1e9,
                      "final_m": r.mavg[-1], "steps": r.steps, "wall_s": round(r.wall_s, 3),
                      "t_ns": [t * 1e9 for t in r.t], "mavg": r.mavg}))


if __name__ == "__main__":
    main()
