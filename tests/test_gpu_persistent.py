"""The persistent batch launch (GRACE_OPT_PERSISTENT): one cooperative kernel takes every
film of an ensemble through all steps of a call, with grid barriers between the y-z and
the x phase of each step.

Its tiles are the grouped path's compile-time bodies, so the result must equal the grouped
launches and the films run alone bit for bit; its barrier waits are bounded, so a missing
arrival (a host-set test hook, no GPU fault) must end in GRACE_ETIMEOUT and leave the
handle usable.  The 2000-step comparison with the oracle is in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import workloads
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()


def _batch(films, opts=None):
    from paper_1411_2565_gb300.grace import GraceBatch
    o = {_lib.OPT_PERSISTENT: 1}
    o.update(opts or {})
    return GraceBatch(films, device=DEV, options=o)


def _m(w):
    return torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).to(DEV)


@pytest.mark.parametrize("steps", [1, 7, 40])
def test_persistent_equals_grouped_and_films_alone(steps):
    from paper_1411_2565_gb300.grace import Grace, GraceBatch
    w = workloads.ensemble(nfilms=16, seed=41)
    p = _batch(w.films)
    p.set_m(_m(w))
    p.step(steps, w.dt)          # 40 steps: two captured graphs of 16, then one direct launch
    p.sync()
    mp = p.get_m()
    g = GraceBatch(w.films, device=DEV, options={_lib.OPT_PERSISTENT: 0})
    g.set_m(_m(w))
    g.step(steps, w.dt)
    assert torch.equal(mp, g.get_m())
    parts = p.split(mp)
    for k in (0, 5, 11):
        f = w.films[k]
        a = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV, tuned=False)
        a.set_hext(f.hext)
        a.set_m(torch.from_numpy(w.m0[k].reshape(-1)).to(DEV))
        a.step(steps, w.dt)
        assert torch.equal(a.get_m().view_as(parts[k]), parts[k]), k
        a.close()
    p.close()
    g.close()


def test_barrier_wait_runs_out_and_is_reported():
    """Block 0 skips its first arrival: every block's wait runs out after 0.2 s, the kernel
    returns, grace_sync reports GRACE_ETIMEOUT once, and with the hook cleared the handle
    steps on normally."""
    w = workloads.ensemble(nfilms=8, seed=43)
    p = _batch(w.films, {_lib.OPT_BARRIER_TIMEOUT_US: 200000})
    p.set_m(_m(w))
    p.step(2, w.dt)
    p.sync()                                             # no failure so far
    p.set_option(_lib.OPT_TEST_SKIP_ARRIVE, 0)
    p.step(3, w.dt)
    with pytest.raises(_lib.GraceError) as e:
        p.sync()
    assert e.value.code == -4                            # GRACE_ETIMEOUT
    p.sync()                                             # reported once, then cleared
    p.set_option(_lib.OPT_TEST_SKIP_ARRIVE, -1)
    p.set_m(_m(w))
    p.step(5, w.dt)
    p.sync()
    _, mavg = p.energy()
    assert np.isfinite(mavg).all()
    # the same five steps on a fresh handle give the same state
    q = _batch(w.films)
    q.set_m(_m(w))
    q.step(5, w.dt)
    assert torch.equal(q.get_m(), p.get_m())
    p.close()
    q.close()


def test_unsupported_shapes_fall_back_to_grouped_launches():
    """A batch with a film thicker than four cells has no persistent body: the option is
    accepted and the grouped launches run (same result as without it)."""
    from paper_1411_2565_gb300.grace import GraceBatch
    f1, m1 = workloads.small_film((32, 16, 6), seed=45)
    f2, m2 = workloads.small_film((64, 16, 1), seed=46)
    m = torch.from_numpy(np.concatenate([m1.reshape(-1), m2.reshape(-1)])).to(DEV)
    outs = []
    for pers in (1, 0):
        g = GraceBatch([f1, f2], device=DEV, options={_lib.OPT_PERSISTENT: pers})
        g.set_m(m)
        g.step(20, 1e-14)
        g.sync()
        outs.append(g.get_m())
        g.close()
    assert torch.equal(outs[0], outs[1])
