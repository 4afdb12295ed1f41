"""Time-dependent applied field (trapezoid envelope of Sec. 5's startTime / decayTime /
stopTime) on the GPU vs the FP64 oracle, through the C ABI.

Bars as for a constant field: one H_eff evaluation max |dH|/Ms <= 1e-5, one step 2e-6 per
component, a trajectory <m> within 1e-4.  Both sides advance the time by repeated FP64
addition of dt, so the envelope's switching decisions agree step for step.
"""
import dataclasses

import numpy as np
import pytest
import torch

import workloads
from oracle import llg
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL_H = 1e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return _lib.load()


def params(f, pulse):
    return llg.Params(f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, np.asarray(f.hext, dtype=np.float64),
                      pulse=pulse)


def make(f, m0, pulse, options=None, hfield=None):
    from paper_1411_2565_gb300.grace import Grace
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV, options=options)
    g.set_hext(f.hext)
    if hfield is not None:
        g.set_hext_field(torch.from_numpy(hfield.reshape(-1)).to(DEV))
    g.set_hext_pulse(pulse)
    g.set_m(torch.from_numpy(m0.reshape(-1)).to(DEV))
    return g


PULSE = (1e-12, 2e-12, 4e-12)


@pytest.mark.parametrize("grid", [(24, 12, 2), (16, 8, 6), (17, 5, 3)])
@pytest.mark.parametrize("t", [0.5e-12, 1.5e-12, 3.1e-12, 5e-12])   # off, full, ramp, after
def test_heff_at_time_matches_oracle(grid, t):
    f, m0 = workloads.small_film(grid, seed=51, Ku=1e4, hext=(4e4, -3e4, 1e4))
    g = make(f, m0, PULSE)
    g.time = t
    h = g.heff().cpu().numpy().reshape(m0.shape)
    ref = llg.heff(m0, params(f, PULSE), t=t)
    assert np.abs(h - ref).max() / f.Ms <= TOL_H


def test_per_cell_field_follows_envelope():
    f, m0 = workloads.small_film((24, 12, 2), seed=52)
    shape = f.shape_zyx
    hf = (5e4 * (2 * workloads.uniform(53, 3 * int(np.prod(shape))) - 1)).astype(np.float32)
    hf = hf.reshape((3,) + shape)
    g = make(f, m0, PULSE, hfield=hf)
    g.time = 3.5e-12
    h = g.heff(_lib.TERM_ZEEMAN).cpu().numpy().reshape(m0.shape)
    p = llg.Params(f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0,
                   hf.astype(np.float64) + np.asarray(f.hext)[:, None, None, None], pulse=PULSE)
    ref = llg.heff(m0, p, mask=llg.ZEEMAN, t=3.5e-12)
    assert np.abs(h - ref).max() / f.Ms <= TOL_H


@pytest.mark.parametrize("integrator", ["euler", "heun"])
def test_film_small_trajectory_through_pulse(integrator):
    """128x32x1 S-state film, 500 steps at dt = 1e-14 s through a 81 mT pulse (on at 1 ps,
    ramp from 2 ps, off at 4 ps): <m> within 1e-4 of the oracle."""
    w = workloads.film_small()
    f, m0 = w.films[0], w.m0[0]
    f = dataclasses.replace(f, hext=(-6.0e4, 2.4e4, 0.0))
    opts = {_lib.OPT_INTEGRATOR: 1} if integrator == "heun" else None
    g = make(f, m0, PULSE, options=opts)
    g.step(w.steps, w.dt)
    mg = g.get_m().cpu().numpy().reshape(m0.shape).astype(np.float64)
    mo = llg.run(m0, params(f, PULSE), w.dt, w.steps, integrator=integrator)
    d = np.abs(mg.reshape(3, -1).mean(1) - mo.reshape(3, -1).mean(1)).max()
    assert d <= 1e-4, d
    assert np.abs(mg - mo).max() <= 1e-3
    # the pulse did something: without it the final state differs
    m_const = llg.run(m0, params(f, None), w.dt, w.steps, integrator=integrator)
    assert np.abs(m_const - mo).max() > 1e-2


@pytest.mark.parametrize("integrator", [0, 1])
def test_single_step_inside_ramp(integrator):
    f, m0 = workloads.small_film((24, 12, 2), seed=54, alpha=0.2, hext=(0.0, 6e4, 0.0))
    g = make(f, m0, PULSE, options={_lib.OPT_INTEGRATOR: integrator})
    g.time = 2.7e-12
    g.step(1, 2e-14)
    m1 = g.get_m().cpu().numpy().reshape(m0.shape)
    step = llg.heun_step if integrator else llg.euler_step
    ref = step(m0, params(f, PULSE), 2e-14, t=2.7e-12)
    assert np.abs(m1 - ref).max() <= 2e-6
    assert g.time == 2.7e-12 + 2e-14


def test_graph_replay_equals_plain_with_pulse():
    f, m0 = workloads.small_film((40, 20, 2), seed=55, alpha=0.3, hext=(5e4, 0.0, 0.0))
    pulse = (3e-14, 2e-13, 5e-13)
    a = make(f, m0, pulse)
    a.step(53, 1e-14)
    b = make(f, m0, pulse, options={_lib.OPT_GRAPH: 0})
    b.step(53, 1e-14)
    assert torch.equal(a.get_m(), b.get_m())
    t = 0.0
    for _ in range(53):
        t = t + 1e-14
    assert a.time == t and b.time == t


def test_time_bookkeeping_and_clearing_the_pulse():
    f, m0 = workloads.small_film((16, 8, 1), seed=56, hext=(2e4, 1e4, 0.0))
    g = make(f, m0, (0.0, 1e-12, 2e-12))
    g.time = 5e-12                                   # after the stop: no applied field
    h_off = g.heff(_lib.TERM_ZEEMAN).cpu().numpy()
    assert np.abs(h_off).max() == 0.0
    g.set_hext_pulse(None)                           # constant field again
    h_on = g.heff(_lib.TERM_ZEEMAN).cpu().numpy().reshape(3, -1)
    assert np.allclose(h_on, np.array([2e4, 1e4, 0.0])[:, None])
    g.step(7, 1e-14)                                 # time advances without an envelope too
    t = 5e-12
    for _ in range(7):
        t = t + 1e-14
    assert g.time == t
    g.set_hext_pulse((0.0, 1.0, 1.0))                # device time resynchronised
    h = g.heff(_lib.TERM_ZEEMAN).cpu().numpy().reshape(3, -1)
    assert np.allclose(h, np.array([2e4, 1e4, 0.0])[:, None])


def test_energy_at_time_matches_oracle():
    f, m0 = workloads.small_film((20, 10, 3), cell=(3e-9, 3e-9, 2e-9), seed=57, Ku=3e4,
                                 hext=(2e4, 1e4, -5e3))
    g = make(f, m0, PULSE)
    g.time = 3.3e-12
    e, _ = g.energy()
    ref = llg.energies(m0, params(f, PULSE), t=3.3e-12)
    scale = max(abs(v) for v in ref[:4])
    assert abs(e["zeeman"] - ref[3]) <= 2e-6 * scale + 1e-6 * abs(ref[3])
    assert abs(e["total"] - ref[4]) <= 2e-6 * scale + 1e-6 * abs(ref[4])


def test_backward_rejects_pulse():
    f, m0 = workloads.small_film((8, 8, 1), seed=58)
    g = make(f, m0, PULSE)
    with pytest.raises(RuntimeError):
        g.backward(torch.zeros(3 * 64, device=DEV), 2, 1e-14)


def test_batch_with_pulse_equals_films_run_alone():
    """The envelope applies to every film of a batch: a batch stepped through a pulse equals
    each film stepped alone with the same pulse, bit for bit."""
    from paper_1411_2565_gb300.grace import GraceBatch
    w = workloads.ensemble(nfilms=6, seed=23)
    pulse = (2e-14, 8e-14, 1.5e-13)
    gb = GraceBatch(w.films, device=DEV)
    gb.set_hext_pulse(pulse)
    gb.set_m(torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).to(DEV))
    gb.step(20, w.dt)
    parts = gb.split(gb.get_m())
    for f, m0, mb in zip(w.films, w.m0, parts):
        g = make(f, m0, pulse)
        g.step(20, w.dt)
        assert torch.equal(g.get_m().view_as(mb), mb)
    f, m0 = w.films[2], w.m0[2]
    mo = llg.run(m0, params(f, pulse), w.dt, 20)
    assert np.abs(parts[2].cpu().numpy().reshape(m0.shape) - mo).max() <= 2e-5
