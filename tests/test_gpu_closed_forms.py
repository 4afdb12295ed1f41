"""The GPU path against textbook closed forms, with no oracle in between (GB300, through
the C ABI).

* Exchange (Sec. 3, six-neighbour stencil with free boundaries): a separable Neumann
  cosine mode m_y = cos(pi a (i+1/2)/nx) cos(pi b (j+1/2)/ny) cos(pi c (k+1/2)/nz) is an
  eigenvector of the discrete Laplacian with eigenvalue
  -sum_d (2 - 2 cos(pi n_d / N_d)) / Delta_d^2, so H_exch = (2A/(mu0 Ms)) lambda m.
* Precession (Eq. 3 with alpha = 0): a single flat cell with x anisotropy in a field
  along x precesses at the Kittel frequency
  omega = gamma0 sqrt((H + H_K + (Ny - Nx) Ms)(H + H_K + (Nz - Nx) Ms)), with the cell's
  self demag factors from Aharoni's prism formula (J. Appl. Phys. 83, 3432 (1998)).
* Macrospin (Eq. 3, explicit Euler): a cubic cell in a field along z follows the
  closed-form damped precession, with first-order convergence in dt.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
MU0 = 4e-7 * math.pi
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return _lib.load()


def aharoni(a, b, c):
    """Demagnetising factor along c of a 2a x 2b x 2c prism (Aharoni 1998, Eq. 1)."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    t = (b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
    t += (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
    t += b / (2 * c) * math.log((ab + a) / (ab - a))
    t += a / (2 * c) * math.log((ab + b) / (ab - b))
    t += c / (2 * a) * math.log((bc - b) / (bc + b))
    t += c / (2 * b) * math.log((ac - a) / (ac + a))
    t += 2 * math.atan(a * b / (c * r))
    t += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    t += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    t += c / (a * b) * (ac + bc)
    t -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return t / math.pi


def cosine_mode(grid, modes):
    nx, ny, nz = grid
    cx = np.cos(math.pi * modes[0] * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(math.pi * modes[1] * (np.arange(ny) + 0.5) / ny)
    cz = np.cos(math.pi * modes[2] * (np.arange(nz) + 0.5) / nz)
    return cz[:, None, None] * cy[None, :, None] * cx[None, None, :]


def laplacian_eigenvalue(grid, modes, cell):
    return -sum((2 - 2 * math.cos(math.pi * k / n)) / (h * h) for n, k, h in zip(grid, modes, cell))


@pytest.mark.parametrize("grid,modes", [((12, 1, 1), (1, 0, 0)), ((12, 1, 1), (5, 0, 0)),
                                        ((16, 10, 3), (3, 2, 1)), ((40, 20, 4), (7, 4, 3)),
                                        ((9, 3, 6), (2, 1, 5)), ((64, 3, 2), (63, 2, 1))])
def test_exchange_of_a_cosine_mode(grid, modes):
    from paper_1411_2565_gb300.grace import Grace
    cell, Ms, A = (3.5e-9, 2.5e-9, 3e-9), 8e5, 1.3e-11
    nx, ny, nz = grid
    m = np.zeros((3, nz, ny, nx), dtype=np.float32)
    m[1] = cosine_mode(grid, modes)
    with Grace(grid, cell, Ms, A, 0.0, 0.1, device=DEV) as g:
        g.set_m(torch.from_numpy(m.reshape(-1)).to(DEV))
        h = g.heff(2).cpu().numpy().reshape(m.shape).astype(np.float64)
    ref = 2 * A / (MU0 * Ms) * laplacian_eigenvalue(grid, modes, cell) * m.astype(np.float64)
    scale = np.abs(ref).max()
    assert np.abs(h - ref).max() <= 1e-5 * max(scale, Ms), (np.abs(h - ref).max(), scale)
    assert np.abs(h[0]).max() == 0.0 and np.abs(h[2]).max() == 0.0


def test_kittel_precession_of_a_flat_cell():
    with open(GOLDEN) as fh:
        mat = json.load(fh)["table1_material"]
    from paper_1411_2565_gb300.grace import Grace
    Ms, HK, A = mat["Ms_A_per_m"], mat["H_anis_A_per_m"], mat["A_J_per_m"]
    Ku = MU0 * Ms * HK / 2
    cell = (100e-9, 100e-9, 2e-9)
    H = 5e4
    nx_, ny_, nz_ = (aharoni(cell[1] / 2, cell[2] / 2, cell[0] / 2),
                     aharoni(cell[0] / 2, cell[2] / 2, cell[1] / 2),
                     aharoni(cell[0] / 2, cell[1] / 2, cell[2] / 2))
    gamma0 = 2.211e5
    w = gamma0 * math.sqrt((H + HK + (ny_ - nx_) * Ms) * (H + HK + (nz_ - nx_) * Ms))
    period = 2 * math.pi / w
    dt = period / 400
    steps = int(12 * period / dt)
    m0 = np.array([1.0, 0.02, 0.0])
    m0 /= np.linalg.norm(m0)
    ys = np.empty(steps)
    with Grace((1, 1, 1), cell, Ms, A, Ku, 0.0, gamma0, device=DEV) as g:
        g.set_hext((H, 0.0, 0.0))
        g.set_m(torch.tensor(m0, dtype=torch.float32, device=DEV))
        traj = torch.empty((steps, 3), dtype=torch.float32, device=DEV)
        for n in range(steps):
            g.step(1, dt)
            g.get_m(out=traj[n])
        ys[:] = traj[:, 1].cpu().numpy()
    up = np.where((ys[:-1] < 0) & (ys[1:] >= 0))[0]
    tc = (up + ys[up] / (ys[up] - ys[up + 1])) * dt
    assert len(tc) >= 10
    measured = (tc[-1] - tc[0]) / (len(tc) - 1)
    assert measured == pytest.approx(period, rel=5e-3)


def test_macrospin_euler_converges_to_the_closed_form():
    """A single cubic cell in H_ext along z (its own demag field -M/3 is parallel to m and
    exerts no torque): tan(theta/2) = tan(theta0/2) exp(-alpha c H t), phi = c H t with
    c = gamma0/(1 + alpha^2).  Explicit Euler is first order: halving dt halves the error."""
    from paper_1411_2565_gb300.grace import Grace
    H, alpha, th0, T, gamma0 = 8e4, 0.2, 1.2, 2e-11, 2.211e5
    c = gamma0 * H / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * c * T))
    ref = np.array([math.sin(th) * math.cos(c * T), math.sin(th) * math.sin(c * T), math.cos(th)])
    errs = []
    for dt in (4e-13, 2e-13):
        with Grace((1, 1, 1), (2e-9, 2e-9, 2e-9), 8e5, 1.3e-11, 0.0, alpha, gamma0, device=DEV) as g:
            g.set_hext((0.0, 0.0, H))
            m0 = [math.sin(th0), 0.0, math.cos(th0)]
            g.set_m(torch.tensor(m0, dtype=torch.float32, device=DEV))
            g.step(int(round(T / dt)), dt)
            m = g.get_m().cpu().numpy().astype(np.float64)
        errs.append(np.abs(m - ref).max())
    assert errs[1] < 2e-2
    assert 1.7 < errs[0] / errs[1] < 2.3, errs
