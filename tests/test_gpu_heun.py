"""Heun (explicit trapezoid) integrator on the GPU vs the FP64 oracle, through the C ABI.

Heun is the higher-order step the paper names as future work (Sec. 6); both sides take
k1 = f(m_n), m* = normalise(m_n + dt k1), k2 = f(m*), m_{n+1} = normalise(m_n + dt (k1+k2)/2).
One step is held to the single-step bar of the Euler path (2e-6 per component); a
trajectory to <m> within 1e-4 of the oracle.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import llg
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
HEUN = {_lib.OPT_INTEGRATOR: 1}


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return _lib.load()


def params(f, ms=None):
    return llg.Params(f.cell, f.Ms if ms is None else ms.astype(np.float64), f.A, f.Ku, f.alpha, f.gamma0,
                      np.asarray(f.hext, dtype=np.float64))


def make(f, m0, options=HEUN, ms=None):
    from paper_1411_2565_gb300.grace import Grace
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV, options=options)
    g.set_hext(f.hext)
    if ms is not None:
        g.set_ms_field(torch.from_numpy(ms.reshape(-1)).to(DEV))
    g.set_m(torch.from_numpy(m0.reshape(-1)).to(DEV))
    return g


# fused fast path, split fast path (nz > 4), generic kernels (odd sizes), one cell
@pytest.mark.parametrize("grid", [(24, 12, 2), (16, 8, 6), (9, 3, 6), (17, 5, 3), (1, 1, 1)])
def test_single_heun_step_matches_oracle(grid):
    f, m0 = workloads.small_film(grid, seed=13, Ku=1e4, alpha=0.2, hext=(0, 2e4, 0))
    g = make(f, m0)
    g.step(1, 2e-14)
    m1 = g.get_m().cpu().numpy().reshape(m0.shape).astype(np.float64)
    ref = llg.heun_step(m0, params(f), 2e-14)
    assert np.abs(m1 - ref).max() <= 2e-6
    assert np.abs(np.sqrt((m1 ** 2).sum(0)) - 1).max() <= 1e-6
    # and it is not the Euler step: the two differ by O(dt^2) terms well above the bar
    eul = llg.euler_step(m0, params(f), 2e-14)
    if grid != (1, 1, 1):
        assert np.abs(ref - eul).max() > 1e-5


def test_heun_step_per_cell_ms():
    f, m0 = workloads.small_film((24, 12, 2), seed=14, Ku=1e4, alpha=0.1)
    ms = (6e5 + 4e5 * workloads.uniform(41, int(np.prod(f.shape_zyx)))).astype(np.float32)
    ms = ms.reshape(f.shape_zyx)
    g = make(f, m0, ms=ms)
    g.step(1, 2e-14)
    m1 = g.get_m().cpu().numpy().reshape(m0.shape)
    ref = llg.heun_step(m0, params(f, ms=ms), 2e-14)
    assert np.abs(m1 - ref).max() <= 2e-6


def test_film_small_heun_trajectory():
    """128x32x1 S-state film, 500 Heun steps at dt = 1e-14 s: <m> within 1e-4 of the oracle."""
    w = workloads.film_small()
    f, m0 = w.films[0], w.m0[0]
    g = make(f, m0)
    g.step(w.steps, w.dt)
    mg = g.get_m().cpu().numpy().reshape(m0.shape).astype(np.float64)
    mo = llg.run(m0, params(f), w.dt, w.steps, integrator="heun")
    d_avg = np.abs(mg.reshape(3, -1).mean(1) - mo.reshape(3, -1).mean(1)).max()
    assert d_avg <= 1e-4, d_avg
    assert np.abs(mg - mo).max() <= 1e-3


def test_heun_graph_replay_equals_plain_launches():
    f, m0 = workloads.small_film((40, 20, 2), seed=15, alpha=0.3)
    a = make(f, m0)
    a.step(37, 1e-14)                 # not a multiple of the graph length
    b = make(f, m0, options={_lib.OPT_INTEGRATOR: 1, _lib.OPT_GRAPH: 0})
    b.step(37, 1e-14)
    assert torch.equal(a.get_m(), b.get_m())


def test_heun_batch_equals_films_run_alone():
    from paper_1411_2565_gb300.grace import GraceBatch
    w = workloads.ensemble(nfilms=6, seed=22)
    gb = GraceBatch(w.films, device=DEV, options=HEUN)
    gb.set_m(torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).to(DEV))
    gb.step(10, w.dt)
    parts = gb.split(gb.get_m())
    for f, m0, mb in zip(w.films, w.m0, parts):
        g = make(f, m0)
        g.step(10, w.dt)
        assert torch.equal(g.get_m().view_as(mb), mb)


def test_heun_rejects_backward():
    f, m0 = workloads.small_film((8, 8, 1), seed=16)
    g = make(f, m0)
    with pytest.raises(RuntimeError):
        g.backward(torch.zeros(3 * 64, device=DEV), 2, 1e-14)


def test_switching_integrator_between_runs():
    """Euler for k steps, then Heun for k steps, equals the oracle doing the same."""
    f, m0 = workloads.small_film((24, 12, 2), seed=17, alpha=0.2)
    g = make(f, m0, options={})
    g.step(5, 1e-14)
    g.set_option(_lib.OPT_INTEGRATOR, 1)
    g.step(5, 1e-14)
    mg = g.get_m().cpu().numpy().reshape(m0.shape)
    p = params(f)
    mo = llg.run(llg.run(m0, p, 1e-14, 5), p, 1e-14, 5, integrator="heun")
    assert np.abs(mg - mo).max() <= 1e-5
