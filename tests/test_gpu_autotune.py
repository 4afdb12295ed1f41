"""Autotuner: every schedule it may pick computes the same result (schedules change the
grouping of work into blocks, not the arithmetic of a line)."""
import os

import numpy as np
import pytest
import torch

import workloads
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu


def test_tuned_schedule_reproduces_default(tmp_path, monkeypatch):
    libbuild.build()
    from paper_1411_2565_gb300 import autotune
    from paper_1411_2565_gb300.grace import Grace
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    w = workloads.film_small()
    f, m0 = w.films[0], w.m0[0]
    opts = autotune.tune([f], [m0], w.dt)
    assert set(opts) == set(autotune.CANDIDATES)
    assert autotune.best([f]) == opts                      # cached
    md = torch.from_numpy(m0.reshape(-1)).cuda()
    ref = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0)
    ref.set_m(md)
    ref.step(40, w.dt)
    for o in ({_lib.OPT_TILE_X: 1, _lib.OPT_TILE_YZ: 1}, {_lib.OPT_TILE_X: 2, _lib.OPT_TILE_YZ: 4},
              opts):
        g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, options=o)
        g.set_m(md)
        g.step(40, w.dt)
        assert torch.equal(g.get_m(), ref.get_m()), o


def test_block_and_ensemble_schedules_match_the_defaults():
    """The shipped schedules of the 256x256x64 block and of an ensemble, and both batch
    groupings, give the library defaults' result bit for bit; so do the two 8-points-per-
    thread z tiles with each other.  The default z schedule of the block (16 points per
    thread, another FFT factorisation) agrees with them to FP32 rounding."""
    libbuild.build()
    from paper_1411_2565_gb300 import autotune
    from paper_1411_2565_gb300.grace import Grace, GraceBatch
    w = workloads.block()
    f, m0 = w.films[0], w.m0[0]
    md = torch.from_numpy(m0.reshape(-1)).cuda()
    ref = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, tuned=False)
    ref.set_m(md)
    ref.step(3, w.dt)
    for o in (autotune.best([f]), {_lib.OPT_TILE_Z: 3}, {_lib.OPT_TILE_Z: 4}, {_lib.OPT_TILE_Z: 0, _lib.OPT_PDL: 0}):
        g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, options=o)
        g.set_m(md)
        g.step(3, w.dt)
        assert torch.equal(g.get_m(), ref.get_m()), o
        g.close()
    outs = []
    for tz in (1, 2):
        g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, options={_lib.OPT_TILE_Z: tz})
        g.set_m(md)
        g.step(3, w.dt)
        outs.append(g.get_m())
        g.close()
    assert torch.equal(outs[0], outs[1])
    assert (outs[0] - ref.get_m()).abs().max().item() <= 1e-6
    ref.close()
    e = workloads.ensemble(nfilms=12, seed=31)
    me = torch.from_numpy(np.concatenate([m.reshape(-1) for m in e.m0])).cuda()
    outs = []
    for o in (None, {_lib.OPT_SIDE_STREAMS: 0}, {_lib.OPT_SIDE_STREAMS: 1, _lib.OPT_GRAPH_STEPS: 8}):
        g = GraceBatch(e.films, options=o, tuned=o is None)
        g.set_m(me)
        g.step(40, e.dt)
        outs.append(g.get_m())
        g.close()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
