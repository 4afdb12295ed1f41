"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to a closed form, an independent formula, an
invariant or a special case with a textbook solution, chosen so that a dropped term,
a wrong sign, a transposed operand or a wrong factor fails at least one of them:

* tensor: cube self term 1/3; Aharoni's closed-form prism factor (J. Appl. Phys. 83,
  3432 (1998)) for the self term and for the body average of whole blocks; direct
  Gauss-Legendre quadrature of the dipole kernel over two cells; far-field convergence.
* demag operator: direct O(N^2) sum vs zero-padded FFT; self-adjointness; E_demag >= 0;
  x<->y mirror symmetry; single cell H = -N M.
* exchange: uniform state gives zero; Neumann cosine modes are eigenvectors with the
  textbook eigenvalue; E_exch >= 0.
* field vs energy: H_eff = -(1/(mu0 Ms V)) dE/dm by central differences of Eq. 1.
* LLG: |m| preserved, m.f = 0, macrospin closed form with first-order Euler convergence,
  Kittel frequency of a flat cell, energy decrease under damping.
* adjoint: central finite differences of the FP64 forward map.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads

from oracle import adjoint as adj
from oracle import demag as dm
from oracle import llg
from oracle.newell import R_SWITCH, asymptotic_tensor, demag_tensor, newell_tensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")
MU0 = 4e-7 * math.pi


def paper():
    with open(GOLDEN) as fh:
        return json.load(fh)


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


def prism_factors(Lx, Ly, Lz):
    return (aharoni(Ly / 2, Lz / 2, Lx / 2), aharoni(Lx / 2, Lz / 2, Ly / 2),
            aharoni(Lx / 2, Ly / 2, Lz / 2))


# ---------------------------------------------------------------- tensor
def test_cube_self_term_is_one_third():
    n = newell_tensor(0.0, 0.0, 0.0, 2e-9, 2e-9, 2e-9)
    assert np.allclose(n[:3], 1.0 / 3.0, rtol=0, atol=1e-14)
    assert np.allclose(n[3:], 0.0, atol=1e-14)


@pytest.mark.parametrize("cell", [(1e-9, 2e-9, 3e-9), (3.90625e-9, 3.90625e-9, 3e-9),
                                  (100e-9, 100e-9, 2e-9), (5e-9, 1e-9, 0.2e-9)])
def test_self_term_matches_aharoni_and_has_unit_trace(cell):
    n = newell_tensor(0.0, 0.0, 0.0, *cell)
    ref = prism_factors(*cell)
    assert np.allclose(n[:3], ref, rtol=1e-11, atol=0)
    assert abs(sum(n[:3]) - 1.0) < 1e-12


def _body_average(grid, cell):
    nx, ny, nz = grid
    ox = np.arange(-(nx - 1), nx)[None, None, :]
    oy = np.arange(-(ny - 1), ny)[None, :, None]
    oz = np.arange(-(nz - 1), nz)[:, None, None]
    w = (nx - np.abs(ox)) * (ny - np.abs(oy)) * (nz - np.abs(oz))
    comps = demag_tensor(ox, oy, oz, cell)
    return [float((w * c).sum()) / (nx * ny * nz) for c in comps]


@pytest.mark.parametrize("grid,cell", [((4, 4, 4), (1e-9, 1e-9, 1e-9)),
                                       ((64, 8, 2), (3.90625e-9, 3.90625e-9, 3e-9)),
                                       ((40, 33, 1), (2e-9, 2e-9, 2e-9))])
def test_body_average_equals_prism_factor(grid, cell):
    """(1/N) sum_ij N(r_i - r_j) is the factor of the whole prism; exercises the far-field
    branch too (offsets beyond the Newell radius for the 64- and 40-cell grids)."""
    avg = _body_average(grid, cell)
    ref = prism_factors(*(n * c for n, c in zip(grid, cell)))
    assert np.allclose(avg[:3], ref, rtol=2e-8, atol=0)
    assert np.allclose(avg[3:], 0.0, atol=1e-12)


def _quadrature_tensor(offset_cells, cell, nodes=24):
    """V E_u[G(r + u)] with u the difference of two uniform points in the cells (tent density),
    G_ab(s) = (delta_ab |s|^2 - 3 s_a s_b)/(4 pi |s|^5); Gauss-Legendre on each half-interval."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    axes = []
    for o, h in zip(offset_cells, cell):
        u = np.concatenate([(x - 1) * h / 2, (x + 1) * h / 2])          # [-h, 0] and [0, h]
        wt = np.concatenate([w, w]) * h / 2 * (1 - np.abs(u) / h) / h
        axes.append((o * h + u, wt))
    sx, sy, sz = np.meshgrid(axes[0][0], axes[1][0], axes[2][0], indexing="ij")
    W = axes[0][1][:, None, None] * axes[1][1][None, :, None] * axes[2][1][None, None, :]
    s = (sx, sy, sz)
    r2 = sx * sx + sy * sy + sz * sz
    r5 = r2 * r2 * np.sqrt(r2)
    V = cell[0] * cell[1] * cell[2]
    out = []
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        g = ((1.0 if a == b else 0.0) * r2 - 3 * s[a] * s[b]) / (4 * math.pi * r5)
        out.append(V * float((W * g).sum()))
    return np.array(out)


@pytest.mark.parametrize("offset", [(2, 0, 0), (2, 1, 1), (0, 3, 1), (3, -2, 0), (-1, 2, -2),
                                    (30, 7, 2), (-26, 11, 3)])
def test_tensor_matches_dipole_quadrature(offset):
    cell = (3.90625e-9, 3.90625e-9, 3e-9)
    ref = _quadrature_tensor(offset, cell)
    got = np.array([float(v) for v in demag_tensor(*offset, cell)])
    scale = np.abs(ref[:3]).max()
    near = max(abs(o) for o in offset) <= R_SWITCH
    # Newell branch: limited by FP64 cancellation (~1e-9 here); asymptotic branch: by the
    # (cell/r)^4 remainder (~3e-7 at 30 cells; a dipole without the correction is ~2e-4 off)
    assert np.max(np.abs(got - ref)) <= (1e-9 if near else 1e-6) * scale


def test_far_field_asymptote_converges_at_fourth_order():
    """Newell minus the corrected asymptote falls like r^-4 relative (r^-2 without the
    correction for non-cubic cells)."""
    cell = (4e-9, 4e-9, 3e-9)
    errs = []
    for d in (6, 12):
        X, Y, Z = d * cell[0], (d // 3) * cell[1], 1 * cell[2]
        nw = np.array(newell_tensor(X, Y, Z, *cell), dtype=float)
        asy = np.array(asymptotic_tensor(X, Y, Z, *cell), dtype=float)
        errs.append(np.abs(nw - asy).max() / np.abs(nw[:3]).max())
    order = math.log2(errs[0] / errs[1])
    assert order > 3.3, errs


def test_tensor_symmetries():
    cell = (2e-9, 3e-9, 1.5e-9)
    for o in [(1, 2, 3), (5, 0, 2), (30, 4, 1)]:
        t = demag_tensor(*o, cell)
        for sx, sy, sz in [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]:
            u = demag_tensor(o[0] * sx, o[1] * sy, o[2] * sz, cell)
            par = [1, 1, 1, sx * sy, sx * sz, sy * sz]
            scale = max(abs(float(v)) for v in t[:3])
            for a, b, p in zip(t, u, par):
                # mirrored offsets round differently inside the 27-point sum
                assert abs(float(b) - p * float(a)) <= 1e-10 * scale


# ---------------------------------------------------------------- demag operator
def _rand_m(shape, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(3,) + shape)
    return v / np.sqrt((v * v).sum(0, keepdims=True))


@pytest.mark.parametrize("grid", [(5, 3, 2), (4, 4, 1), (1, 1, 1), (3, 1, 1), (2, 5, 3)])
def test_fft_convolution_equals_direct_sum(grid):
    nx, ny, nz = grid
    cell = (3e-9, 2e-9, 4e-9)
    m = _rand_m((nz, ny, nx), 1)
    Ms = 8e5 * (1 + 0.3 * np.random.default_rng(2).random((nz, ny, nx)))
    hd = dm.demag_direct(m, Ms, cell)
    hf = dm.demag_fft(m, Ms, cell)
    assert np.max(np.abs(hd - hf)) <= 1e-12 * np.max(np.abs(hd))


def test_direct_sum_far_branch_equals_fft():
    """A grid longer than the Newell radius: both paths see the asymptotic branch."""
    cell = (2e-9, 2e-9, 2e-9)
    m = _rand_m((1, 2, 60), 3)
    hf = dm.demag_fft(m, 1e6, cell)
    cells = [(0, 0, 0), (59, 1, 0), (30, 0, 0)]
    hs = dm.demag_at(cells, m, 1e6, cell)
    for k, (x, y, z) in enumerate(cells):
        assert np.allclose(hs[k], hf[:, z, y, x], rtol=0, atol=1e-10 * 1e6)


def test_single_cell_field_is_minus_self_tensor_times_m():
    cell = (5e-9, 3e-9, 2e-9)
    m = np.array([0.3, -0.5, 0.8])[:, None, None, None]
    m = m / np.linalg.norm(m)
    n = newell_tensor(0, 0, 0, *cell)
    h = dm.demag_fft(m, 1e6, cell)[:, 0, 0, 0]
    assert np.allclose(h, -1e6 * np.array(n[:3]) * m[:, 0, 0, 0], rtol=1e-12)


def test_demag_is_self_adjoint_and_energy_positive():
    cell = (3e-9, 3e-9, 2e-9)
    a = _rand_m((3, 6, 7), 4)
    b = _rand_m((3, 6, 7), 5)
    D = llg.Demag((7, 6, 3), cell)
    lhs = float((a * D(b, 1.0)).sum())
    rhs = float((D(a, 1.0) * b).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert float((a * D(a, 1.0)).sum()) < 0.0        # -m.N m < 0  <=>  E_demag > 0


def test_demag_mirror_symmetry_x_y():
    cell = (3e-9, 2e-9, 4e-9)
    m = _rand_m((2, 3, 5), 6)
    h = dm.demag_fft(m, 1e6, cell)
    ms = np.stack([m[1], m[0], m[2]]).transpose(0, 1, 3, 2)
    hs = dm.demag_fft(ms, 1e6, (cell[1], cell[0], cell[2]))
    back = np.stack([hs[1], hs[0], hs[2]]).transpose(0, 1, 3, 2)
    assert np.allclose(back, h, rtol=0, atol=1e-12 * np.abs(h).max())


# ---------------------------------------------------------------- exchange
def test_exchange_of_uniform_state_is_zero():
    m = np.zeros((3, 3, 4, 5))
    m[0] = 0.6
    m[2] = 0.8
    p = llg.Params((2e-9, 3e-9, 4e-9), 8e5, 1.3e-11, 0.0, 0.1)
    assert np.abs(llg.exchange_field(m, p)).max() == 0.0


@pytest.mark.parametrize("j", [1, 2, 5])
def test_neumann_cosine_mode_is_eigenvector(j):
    nx, h = 12, 2e-9
    i = np.arange(nx) + 0.5
    mode = np.cos(math.pi * j * i / nx)
    m = np.zeros((3, 1, 1, nx))
    m[1, 0, 0] = mode
    lap = llg.laplacian(m, (h, h, h))
    lam = -(2 - 2 * math.cos(math.pi * j / nx)) / h ** 2
    assert np.allclose(lap[1, 0, 0], lam * mode, rtol=0, atol=1e-10 * abs(lam))


def test_field_is_minus_energy_gradient():
    """H_eff,i = -(1/(mu0 Ms_i V)) dE/dm_i (central differences of Eq. 1 energies)."""
    cell = (3e-9, 2.5e-9, 2e-9)
    grid = (4, 3, 2)
    m = _rand_m((2, 3, 4), 7)
    Ms = 6e5 + 4e5 * np.random.default_rng(8).random((2, 3, 4))
    p = llg.Params(cell, Ms, 1.3e-11, 4e4, 0.1, hext=(1e4, -2e4, 3e4))
    D = llg.Demag(grid, cell)
    H = llg.heff(m, p, D)
    V = cell[0] * cell[1] * cell[2]
    for (c, z, y, x) in [(0, 0, 0, 0), (1, 1, 2, 3), (2, 0, 1, 2), (0, 1, 1, 1)]:
        e = 1e-6
        mp = m.copy()
        mp[c, z, y, x] += e
        mm = m.copy()
        mm[c, z, y, x] -= e
        dE = (llg.energies(mp, p, D)[4] - llg.energies(mm, p, D)[4]) / (2 * e)
        h_fd = -dE / (MU0 * Ms[z, y, x] * V)
        assert h_fd == pytest.approx(H[c, z, y, x], rel=1e-6, abs=1e-6 * np.abs(H).max())


# ---------------------------------------------------------------- LLG + Euler
def test_llg_torque_is_orthogonal_and_step_keeps_unit_length():
    cell = (3e-9, 3e-9, 3e-9)
    m = _rand_m((2, 4, 5), 9)
    p = llg.Params(cell, 8e5, 1.3e-11, 1e4, 0.3, hext=(1e4, 0, 0))
    H = llg.heff(m, p)
    f = llg.llg_rhs(m, H, p.alpha, p.gamma0)
    assert np.abs((m * f).sum(0)).max() <= 1e-12 * np.abs(f).max()
    m1 = llg.run(m, p, 1e-14, 5)
    assert np.abs(np.sqrt((m1 * m1).sum(0)) - 1).max() < 1e-14


def _macrospin(dt, steps, alpha, H, theta0, phi0=0.0, integrator="euler", pulse=None):
    cell = (2e-9, 2e-9, 2e-9)
    m0 = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0),
                   math.cos(theta0)])[:, None, None, None]
    p = llg.Params(cell, 8e5, 1.3e-11, 0.0, alpha, hext=(0.0, 0.0, H), pulse=pulse)
    return llg.run(m0, p, dt, steps, llg.Demag((1, 1, 1), cell), integrator=integrator)[:, 0, 0, 0], p


def _pulse_area(T, t0, t1, t2):
    """Integral over [0, T] of the trapezoid envelope (0 | 1 from t0 | linear 1 -> 0 on [t1, t2])."""
    if T <= t0:
        return 0.0
    if T <= t1:
        return T - t0
    if T <= t2:
        r = T - t1
        return (t1 - t0) + r - r * r / (2 * (t2 - t1))
    return (t1 - t0) + 0.5 * (t2 - t1)


def _macrospin_exact(H, alpha, th0, area, gamma0=2.211e5):
    """Macrospin in H(t) z: phi = g/(1+a^2) int H, tan(theta/2) decays by exp(-a g/(1+a^2) int H)."""
    c = gamma0 * H / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * c * area))
    ph = c * area
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def test_macrospin_closed_form_first_order():
    """Single cubic cell: its demag field -M/3 is parallel to m (no torque), so in H_ext || z
    tan(theta/2) = tan(theta0/2) exp(-alpha g H t/(1+alpha^2)), phi = phi0 + g H t/(1+alpha^2)."""
    H, alpha, th0, T = 8e4, 0.2, 1.2, 2e-11
    errs = []
    for dt in (4e-13, 2e-13):
        steps = int(round(T / dt))
        m, p = _macrospin(dt, steps, alpha, H, th0)
        c = p.gamma0 * H / (1 + alpha ** 2)
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * c * T))
        ph = c * T
        ref = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        errs.append(np.abs(m - ref).max())
    assert errs[1] < 2e-2
    assert 1.7 < errs[0] / errs[1] < 2.3, errs


def test_heun_macrospin_second_order():
    """The Heun integrator on the macrospin closed form: error falls ~4x when dt halves."""
    H, alpha, th0, T = 8e4, 0.2, 1.2, 2e-11
    errs = []
    for dt in (8e-13, 4e-13):
        steps = int(round(T / dt))
        m, p = _macrospin(dt, steps, alpha, H, th0, integrator="heun")
        c = p.gamma0 * H / (1 + alpha ** 2)
        th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * c * T))
        ph = c * T
        ref = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        errs.append(np.abs(m - ref).max())
    assert errs[1] < 5e-4
    assert 3.3 < errs[0] / errs[1] < 4.7, errs


@pytest.mark.parametrize("T", [1.6e-11, 2.4e-11])        # inside the ramp, after the stop
def test_pulsed_field_macrospin_euler(T):
    """Trapezoid field pulse (off until 2 ps, full until 8 ps, linear to zero at 20 ps) on the
    macrospin: the exact solution depends on the pulse only through its area up to T.  Euler
    samples the field at the start of each step, so with the edges on step boundaries its
    error is first order (ratio ~2 per halving) and small."""
    H, alpha, th0, pulse = 1.2e5, 0.2, 1.2, (2e-12, 8e-12, 2e-11)
    ref = _macrospin_exact(H, alpha, th0, _pulse_area(T, *pulse))
    errs = []
    for dt in (2e-13, 1e-13):
        m, _ = _macrospin(dt, int(round(T / dt)), alpha, H, th0, pulse=pulse)
        errs.append(np.abs(m - ref).max())
    assert errs[1] < 2e-2
    assert 1.7 < errs[0] / errs[1] < 2.3, errs


@pytest.mark.parametrize("T", [1.6e-11, 2.4e-11])
def test_pulsed_field_macrospin_heun_second_order(T):
    """Heun on a pulse that is on from t = 0 and ramps down linearly from 8 ps to 20 ps:
    the envelope is continuous with kinks on step boundaries, so the trapezoid rule in
    time keeps second order (ratio ~4 per halving).  A corrector that sampled the field at
    t_n instead of t_n + dt would fall to first order inside the ramp."""
    H, alpha, th0, pulse = 1.2e5, 0.2, 1.2, (0.0, 8e-12, 2e-11)
    ref = _macrospin_exact(H, alpha, th0, _pulse_area(T, *pulse))
    errs = []
    for dt in (4e-13, 2e-13):
        m, _ = _macrospin(dt, int(round(T / dt)), alpha, H, th0, integrator="heun", pulse=pulse)
        errs.append(np.abs(m - ref).max())
    assert errs[1] < 5e-4
    assert 3.3 < errs[0] / errs[1] < 4.7, errs


def test_euler_samples_field_at_step_start():
    """Explicit Euler takes f(t_n, m_n): with the pulse switching on exactly at t = dt the
    first step sees no field (m unchanged), and the second step is one Euler step of the
    constant-field macrospin."""
    dt, H, alpha, th0 = 1e-13, 1e5, 0.1, 0.9
    pulse = (dt, 1.0, 1.0)
    m1, _ = _macrospin(dt, 1, alpha, H, th0, pulse=pulse)
    m0 = np.array([math.sin(th0), 0.0, math.cos(th0)])
    assert np.abs(m1 - m0).max() < 1e-14
    m2, _ = _macrospin(dt, 2, alpha, H, th0, pulse=pulse)
    c = 2.211e5 / (1 + alpha ** 2)
    h = np.array([0.0, 0.0, H])
    u = m0 - dt * c * (np.cross(m0, h) + alpha * np.cross(m0, np.cross(m0, h)))
    assert np.abs(m2 - u / np.linalg.norm(u)).max() < 1e-12


def test_pulse_off_leaves_macrospin_still():
    """Before t_start the applied field is zero and a cube's own demag field is parallel to
    m, so nothing moves."""
    m, _ = _macrospin(1e-13, 50, 0.1, 1e5, 0.9, phi0=0.4, pulse=(1e-11, 2e-11, 3e-11))
    ref = np.array([math.sin(0.9) * math.cos(0.4), math.sin(0.9) * math.sin(0.4), math.cos(0.9)])
    assert np.abs(m - ref).max() < 1e-14


def test_kittel_frequency_of_flat_cell():
    """Undamped precession about x of a single flat cell with x anisotropy (Table 1 material):
    omega = g sqrt((H + H_K + (Ny - Nx) Ms)(H + H_K + (Nz - Nx) Ms))."""
    mat = paper()["table1_material"]
    Ms, HK = mat["Ms_A_per_m"], mat["H_anis_A_per_m"]
    Ku = MU0 * Ms * HK / 2
    cell = (100e-9, 100e-9, 2e-9)
    H = 5e4
    p = llg.Params(cell, Ms, mat["A_J_per_m"], Ku, 0.0, hext=(H, 0.0, 0.0))
    n = newell_tensor(0, 0, 0, *cell)
    w = p.gamma0 * math.sqrt((H + HK + (n[1] - n[0]) * Ms) * (H + HK + (n[2] - n[0]) * Ms))
    period = 2 * math.pi / w
    dt = period / 400
    steps = int(12 * period / dt)
    m0 = np.array([1.0, 0.02, 0.0])[:, None, None, None]
    m0 /= np.linalg.norm(m0)
    D = llg.Demag((1, 1, 1), cell)
    m, ys = m0, []
    for _ in range(steps):
        m = llg.euler_step(m, p, dt, D)
        ys.append(m[1, 0, 0, 0])
    ys = np.array(ys)
    up = np.where((ys[:-1] < 0) & (ys[1:] >= 0))[0]
    tc = (up + ys[up] / (ys[up] - ys[up + 1])) * dt
    measured = (tc[-1] - tc[0]) / (len(tc) - 1)
    assert len(tc) >= 10
    assert measured == pytest.approx(period, rel=5e-3)


def test_energy_decreases_under_damping():
    cell = (3e-9, 3e-9, 3e-9)
    m = llg.normalise(_rand_m((2, 4, 6), 10) + np.array([2.0, 0, 0])[:, None, None, None])
    p = llg.Params(cell, 8e5, 1.3e-11, 1e4, 0.5)
    D = llg.Demag((6, 4, 2), cell)
    e_prev = llg.energies(m, p, D)[4]
    for _ in range(40):
        m = llg.euler_step(m, p, 2e-14, D)
        e = llg.energies(m, p, D)[4]
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e


# ---------------------------------------------------------------- adjoint
def test_adjoint_matches_central_differences():
    grid = (6, 4, 2)
    cell = (4e-9, 4e-9, 3e-9)
    m0 = _rand_m((2, 4, 6), 11)
    target = _rand_m((2, 4, 6), 12)
    Ms = np.full((2, 4, 6), 8e5)
    hx = np.zeros((3, 2, 4, 6))
    hx[0] = 1e4
    p = llg.Params(cell, Ms, 1.3e-11, 2e3, 0.1, hext=hx)
    D = llg.Demag(grid, cell)
    dt, steps = 2e-14, 12
    loss, g_m0, g_h, g_ms = adj.gradients(m0, p, dt, steps, target, D)

    def L(m0_=m0, Ms_=Ms, hx_=hx):
        q = llg.Params(cell, Ms_, 1.3e-11, 2e3, 0.1, hext=hx_)
        return adj.loss_mse(llg.run(m0_, q, dt, steps, D), target)

    assert L() == pytest.approx(loss, rel=1e-14)
    for (c, z, y, x) in [(0, 0, 0, 0), (1, 1, 2, 3), (2, 0, 3, 5)]:
        h = 1e-3 * 1e4
        hp, hm = hx.copy(), hx.copy()
        hp[c, z, y, x] += h
        hm[c, z, y, x] -= h
        fd = (L(hx_=hp) - L(hx_=hm)) / (2 * h)
        assert fd == pytest.approx(g_h[c, z, y, x], rel=1e-5, abs=1e-6 * np.abs(g_h).max())
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (0, 3, 5)]:
        h = 1e-3 * Ms[z, y, x]
        mp, mm = Ms.copy(), Ms.copy()
        mp[z, y, x] += h
        mm[z, y, x] -= h
        fd = (L(Ms_=mp) - L(Ms_=mm)) / (2 * h)
        assert fd == pytest.approx(g_ms[z, y, x], rel=1e-5, abs=1e-6 * np.abs(g_ms).max())
    v = _rand_m((2, 4, 6), 13)
    e = 1e-6
    fd = (L(m0_=m0 + e * v) - L(m0_=m0 - e * v)) / (2 * e)
    assert fd == pytest.approx(float((g_m0 * v).sum()), rel=1e-6)


def test_adjoint_step_dot_product():
    """<J v, w> = <v, J^T w> for one step m' = normalise(m + dt f(m, H(m))) with every term
    on (per-cell Ms, anisotropy, per-cell field): J v by central differences of the FP64
    step, J^T w from the oracle's adjoint step, for random directions v and w."""
    grid, cell = (6, 4, 2), (4e-9, 4e-9, 3e-9)
    m = _rand_m((2, 4, 6), 21)
    Ms = 6e5 + 4e5 * workloads.uniform(22, 48).reshape(2, 4, 6)
    hx = 2e4 * (2 * workloads.uniform(23, 144).reshape(3, 2, 4, 6) - 1)
    p = llg.Params(cell, Ms, 1.3e-11, 3e4, 0.15, hext=hx)
    D = llg.Demag(grid, cell)
    dt = 3e-14
    v = workloads.gaussian(24, 144).reshape(3, 2, 4, 6)
    w = workloads.gaussian(25, 144).reshape(3, 2, 4, 6)
    e = 1e-6
    jv = (llg.euler_step(m + e * v, p, dt, D) - llg.euler_step(m - e * v, p, dt, D)) / (2 * e)
    jtw, _, _ = adj.adjoint_step(m, w, p, dt, D)
    lhs, rhs = float((jv * w).sum()), float((v * jtw).sum())
    assert lhs == pytest.approx(rhs, rel=1e-8)
