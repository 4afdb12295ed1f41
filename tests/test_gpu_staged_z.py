"""The z pass whose blocks stage the next tile's spectrum columns into shared memory with a
TMA tensor copy (GRACE_OPT_TILE_Z = 4, one film with a padded z length of 128).

It runs the same arithmetic as the default 16-points-per-thread z pass, so the two must
agree bit for bit (and, through test_z_schedules_match_oracle, with the FP64 oracle).  Its
wait for each copy is bounded: a block that skips its first copy (a host-set test hook,
no GPU fault) must end in GRACE_ETIMEOUT, reported once, with the handle usable after."""
import numpy as np
import pytest
import torch

import workloads
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
STAGED = {_lib.OPT_TILE_Z: 4}


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()


def _film(grid, seed):
    return workloads.small_film(grid, cell=(3e-9, 3e-9, 3e-9), seed=seed, Ku=1e4, hext=(1e4, -5e3, 2e3))


def _handle(f, opts):
    from paper_1411_2565_gb300.grace import Grace
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV, options=opts)
    g.set_hext(f.hext)
    return g


@pytest.mark.parametrize("grid", [(24, 20, 33), (40, 9, 64), (64, 64, 48)])
def test_staged_z_equals_default_z(grid):
    f, m0 = _film(grid, seed=61)
    m = torch.from_numpy(m0.reshape(-1)).to(DEV)
    out = []
    for opts in ({_lib.OPT_TILE_Z: 3}, STAGED):
        g = _handle(f, opts)
        g.set_m(m)
        h = g.heff().clone()
        g.step(6, 1e-14)
        out.append((h, g.get_m()))
        g.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])


def test_staged_z_copy_wait_runs_out_and_is_reported():
    """Block 0 skips its first copy: its wait runs out after 0.05 s, it records
    GRACE_ETIMEOUT and leaves the kernel; grace_sync reports it once; with the hook
    cleared the handle steps on and matches a fresh handle bit for bit."""
    f, m0 = _film((24, 20, 33), seed=62)
    m = torch.from_numpy(m0.reshape(-1)).to(DEV)
    g = _handle(f, {**STAGED, _lib.OPT_BARRIER_TIMEOUT_US: 50000})
    g.set_m(m)
    g.step(2, 1e-14)
    g.sync()                                             # no failure so far
    g.set_option(_lib.OPT_TEST_SKIP_ARRIVE, 0)
    g.step(1, 1e-14)
    with pytest.raises(_lib.GraceError) as e:
        g.sync()
    assert e.value.code == -4                            # GRACE_ETIMEOUT
    g.sync()                                             # reported once, then cleared
    g.set_option(_lib.OPT_TEST_SKIP_ARRIVE, -1)
    g.set_m(m)
    g.step(5, 1e-14)
    g.sync()
    _, mavg = g.energy()
    assert np.isfinite(mavg).all()
    q = _handle(f, STAGED)
    q.set_m(m)
    q.step(5, 1e-14)
    assert torch.equal(q.get_m(), g.get_m())
    g.close()
    q.close()
