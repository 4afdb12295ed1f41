"""Standard-problem-4-shaped reversal (Sec. 4) on the GPU: relaxation into the S-state at
alpha = 0.5, then reversal at alpha = 0.02 under field 1 and field 2, on 500 x 125 x 3 nm
at two discretisations (128 x 32 and 256 x 64 cells).  No external reference curve is
available, so the checks are self-consistency: the FP64 oracle over the first 2000 steps
of the relaxation and of the reversal (<m> within 1e-4), and the two discretisations
against each other (first zero of <m_x> within 2 %, <m>(t) curves within 0.08, the
relaxed states within 2e-3; second-order spatial error makes the coarse-fine gap about
three quarters of the coarse grid's own error)."""
import numpy as np
import pytest

import workloads
from oracle import llg
from paper_1411_2565_gb300 import build as libbuild
from paper_1411_2565_gb300 import mumag4 as M

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GRIDS = [(128, 32), (256, 64)]


@pytest.fixture(scope="module")
def relaxed():
    libbuild.build()
    out = {}
    for g in GRIDS:
        m0 = workloads.near_saturated_m((1, g[1], g[0]), (1.0, 1.0, 1.0), seed=10)
        out[g] = M.relax(g, m0, 2e-9, device=DEV)
    return out


@pytest.fixture(scope="module")
def reversals(relaxed):
    return {(g, k): M.reverse(g, relaxed[g], k, 1e-9, 1e-12, device=DEV) for g in GRIDS for k in (1, 2)}


def _params(grid, alpha, hext, pulse=None):
    return llg.Params(M.cell_size(grid), M.MS, M.A_EX, 0.0, alpha, 2.211e5, np.asarray(hext, dtype=np.float64),
                      pulse=pulse)


def test_relaxation_start_matches_oracle():
    libbuild.build()
    g = GRIDS[0]
    m0 = workloads.near_saturated_m((1, g[1], g[0]), (1.0, 1.0, 1.0), seed=10)
    dt = M.time_step(g)
    mg = M.relax(g, m0, 2000 * dt, device=DEV)
    mo = llg.run(m0, _params(g, 0.5, (0.0, 0.0, 0.0)), dt, 2000)
    assert np.abs(mg.reshape(3, -1).mean(1) - mo.reshape(3, -1).mean(1)).max() <= 1e-4
    assert np.abs(mg - mo).max() <= 1e-3


def test_reversal_start_matches_oracle(relaxed):
    g = GRIDS[0]
    dt = M.time_step(g)
    r = M.reverse(g, relaxed[g], 1, 2000 * dt, 200 * dt, device=DEV)
    mo = llg.run(relaxed[g], _params(g, 0.02, M.field_Apm(1), (0.0, 2000 * dt, 4000 * dt)), dt, 2000)
    assert np.abs(np.asarray(r.mavg[-1]) - mo.reshape(3, -1).mean(1)).max() <= 1e-4
    assert np.abs(r.m_final - mo).max() <= 1e-3


def test_relaxed_s_state_agrees_between_discretisations(relaxed):
    a, b = (relaxed[g].reshape(3, -1).astype(np.float64).mean(1) for g in GRIDS)
    assert np.abs(a - b).max() <= 2e-3
    assert a[0] > 0.9 and abs(a[2]) < 1e-3        # in-plane, mostly along +x


@pytest.mark.parametrize("field_no", [1, 2])
def test_reversal_agrees_between_discretisations(reversals, field_no):
    rc, rf = reversals[(GRIDS[0], field_no)], reversals[(GRIDS[1], field_no)]
    assert rc.t_cross is not None and rf.t_cross is not None
    assert abs(rc.t_cross - rf.t_cross) <= 0.02 * rf.t_cross
    assert M.curve_distance(rc, rf) <= 0.08
    for r in (rc, rf):
        assert r.mavg[-1][0] < -0.9                  # reversed after 1 ns
        n = np.sqrt((r.m_final.astype(np.float64) ** 2).sum(0))
        assert np.abs(n - 1).max() <= 1e-5
