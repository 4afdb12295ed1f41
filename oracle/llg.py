"""Effective field, LLG right-hand side, explicit Euler step and energies, FP64.

Follows the paper's Sec. 2 (Eqs. 1-3) and Sec. 3 (six-neighbour exchange, explicit
Euler), with these readings where the text is garbled or silent:

* Eq. 1's exchange term repeats (grad M_x/Ms)^2 three times; read as the sum over the
  three components.  Eq. 2 lacks the 1/mu0: H_eff = -(1/mu0) dE/dM, so
  H_exch = (2A/(mu0 Ms)) lap m and H_anis = (2Ku/(mu0 Ms)) m_x x.
* The discrete Laplacian is the six-neighbour sum of (m_j - m_i)/d^2 per axis with free
  (Neumann) boundaries: a missing neighbour contributes nothing.  With a per-cell Ms the
  observer cell's Ms enters the exchange and anisotropy prefactors.
* Eq. 3's gamma multiplies mu0 H; gamma0 = mu0 gamma = 2.211e5 m/(A s) is applied to H
  in A/m.  In unit-vector form dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)].
* Euler uses H from m_n; m_{n+1} = normalise(m_n + dt f(m_n)).
* Energies (Eq. 1 times the cell volume V): E_exch = A V sum_bonds |m_j - m_i|^2/d^2,
  E_anis = Ku V sum (1 - m_x^2), E_demag = -(mu0/2) V sum Ms m.H_d,
  E_zeeman = -mu0 V sum Ms m.H_ext.
* Time-dependent applied field (the input file's startTime / decayTime / stopTime,
  Sec. 5, whose meaning the paper leaves open): H_ext(r, t) = s(t) H_ext(r) with s = 0
  before t_start, 1 until t_decay, falling linearly to 0 at t_stop and 0 afterwards.
  Euler evaluates the field at t_n; Heun's corrector at t_n + dt.  Time advances by
  repeated addition t <- t + dt from t_0.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from .demag import demag_direct, demag_fft, padded_tensor_spectrum
from .newell import R_SWITCH

MU0 = 4e-7 * np.pi

DEMAG, EXCH, ANIS, ZEEMAN = 1, 2, 4, 8
ALL_TERMS = DEMAG | EXCH | ANIS | ZEEMAN


@dataclass
class Params:
    """Film parameters: cell (m), Ms (scalar or [nz][ny][nx]), A, Ku (x axis), alpha, gamma0,
    hext (3-vector or [3][nz][ny][nx], A/m)."""
    cell: Sequence[float]
    Ms: object
    A: float
    Ku: float
    alpha: float
    gamma0: float = 2.211e5
    hext: object = (0.0, 0.0, 0.0)
    r_switch: int = R_SWITCH
    pulse: Optional[Sequence[float]] = None     # (t_start, t_decay, t_stop) in s, or constant


def field_scale(t: float, pulse) -> float:
    """Envelope s(t) of the applied field: 0 before t_start, 1 until t_decay, linear to 0
    at t_stop, 0 after; 1 for a constant field (pulse None)."""
    if pulse is None:
        return 1.0
    t0, t1, t2 = pulse
    if t < t0:
        return 0.0
    if t < t1:
        return 1.0
    if t < t2:
        return (t2 - t) / (t2 - t1)
    return 0.0


def laplacian(m, cell):
    """Six-neighbour Laplacian sum_d sum_{j in nbr_d(i)} (m_j - m_i)/d^2, Neumann boundaries."""
    m = np.asarray(m, dtype=np.float64)
    out = np.zeros_like(m)
    for axis, h in ((3, cell[0]), (2, cell[1]), (1, cell[2])):
        if m.shape[axis] < 2:
            continue
        d = np.diff(m, axis=axis) / (h * h)          # (m_{i+1} - m_i)/h^2 on each bond
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        out[tuple(lo)] += d          # cell i sees +(m_{i+1} - m_i)
        out[tuple(hi)] -= d          # cell i+1 sees +(m_i - m_{i+1})
    return out


def exchange_field(m, p: Params):
    return 2.0 * p.A / (MU0 * np.asarray(p.Ms, dtype=np.float64)) * laplacian(m, p.cell)


def anisotropy_field(m, p: Params):
    h = np.zeros_like(np.asarray(m, dtype=np.float64))
    h[0] = 2.0 * p.Ku / (MU0 * np.asarray(p.Ms, dtype=np.float64)) * m[0]
    return h


def zeeman_field(m, p: Params, t: float = 0.0):
    h = field_scale(t, p.pulse) * np.asarray(p.hext, dtype=np.float64)
    if h.ndim == 1:
        return np.broadcast_to(h[:, None, None, None], np.shape(m)).copy()
    return h.copy()


class Demag:
    """Demag operator for one grid; caches the padded tensor spectrum (FFT) or uses the direct sum."""

    def __init__(self, grid, cell, method: str = "fft", r_switch: int = R_SWITCH):
        self.grid, self.cell, self.method, self.r_switch = tuple(grid), tuple(cell), method, r_switch
        self.spectrum = (padded_tensor_spectrum(self.grid, cell, r_switch)
                         if method == "fft" else None)

    def __call__(self, m, Ms):
        if self.method == "fft":
            return demag_fft(m, Ms, self.cell, self.spectrum)
        return demag_direct(m, Ms, self.cell, self.r_switch)


def heff(m, p: Params, demag: Optional[Demag] = None, mask: int = ALL_TERMS, t: float = 0.0):
    """H_eff of Eq. 2 at time t restricted to the terms in ``mask`` (A/m), layout [3][nz][ny][nx]."""
    m = np.asarray(m, dtype=np.float64)
    h = np.zeros_like(m)
    if mask & DEMAG:
        if demag is None:
            _, nz, ny, nx = m.shape
            demag = Demag((nx, ny, nz), p.cell, "fft", p.r_switch)
        h += demag(m, p.Ms)
    if mask & EXCH:
        h += exchange_field(m, p)
    if mask & ANIS:
        h += anisotropy_field(m, p)
    if mask & ZEEMAN:
        h += zeeman_field(m, p, t)
    return h


def llg_rhs(m, H, alpha, gamma0):
    """Eq. 3 divided by Ms: -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)]."""
    mxh = np.cross(m, H, axis=0)
    return -gamma0 / (1.0 + alpha * alpha) * (mxh + alpha * np.cross(m, mxh, axis=0))


def normalise(v):
    return v / np.sqrt((v * v).sum(axis=0, keepdims=True))


def euler_step(m, p: Params, dt: float, demag: Optional[Demag] = None, t: float = 0.0):
    """m_{n+1} = normalise(m_n + dt f(m_n, H_eff(m_n, t_n)))."""
    m = np.asarray(m, dtype=np.float64)
    return normalise(m + dt * llg_rhs(m, heff(m, p, demag, t=t), p.alpha, p.gamma0))


def heun_step(m, p: Params, dt: float, demag: Optional[Demag] = None, t: float = 0.0):
    """Explicit trapezoid (Heun) with renormalisation, the higher-order integrator the paper
    names as future work (Sec. 6): k1 = f(m_n, t_n), m* = normalise(m_n + dt k1),
    k2 = f(m*, t_n + dt), m_{n+1} = normalise(m_n + dt (k1 + k2)/2)."""
    m = np.asarray(m, dtype=np.float64)
    k1 = llg_rhs(m, heff(m, p, demag, t=t), p.alpha, p.gamma0)
    ms = normalise(m + dt * k1)
    k2 = llg_rhs(ms, heff(ms, p, demag, t=t + dt), p.alpha, p.gamma0)
    return normalise(m + 0.5 * dt * (k1 + k2))


def run(m0, p: Params, dt: float, steps: int, demag: Optional[Demag] = None, keep=False,
        integrator: str = "euler", t0: float = 0.0):
    """Take ``steps`` steps (Euler or Heun) from time t0; returns the final state (and every
    state if ``keep``)."""
    m = np.asarray(m0, dtype=np.float64)
    if demag is None:
        _, nz, ny, nx = m.shape
        demag = Demag((nx, ny, nz), p.cell, "fft", p.r_switch)
    step = heun_step if integrator == "heun" else euler_step
    states = [m] if keep else None
    t = float(t0)
    for _ in range(steps):
        m = step(m, p, dt, demag, t)
        t = t + dt
        if keep:
            states.append(m)
    return (m, states) if keep else m


def energies(m, p: Params, demag: Optional[Demag] = None, t: float = 0.0):
    """(E_exch, E_anis, E_demag, E_zeeman, E_total) in joules at time t, from Eq. 1 times V
    per cell."""
    m = np.asarray(m, dtype=np.float64)
    dx, dy, dz = p.cell
    V = dx * dy * dz
    Ms = np.asarray(p.Ms, dtype=np.float64)
    e_ex = 0.0
    for axis, h in ((3, dx), (2, dy), (1, dz)):
        if m.shape[axis] > 1:
            d = np.diff(m, axis=axis)
            e_ex += p.A * V * np.sum(d * d) / (h * h)
    e_an = p.Ku * V * np.sum(1.0 - m[0] ** 2)
    hd = heff(m, p, demag, DEMAG)
    e_d = -0.5 * MU0 * V * np.sum(Ms * (m * hd).sum(axis=0))
    hz = zeeman_field(m, p, t)
    e_z = -MU0 * V * np.sum(Ms * (m * hz).sum(axis=0))
    return e_ex, e_an, e_d, e_z, e_ex + e_an + e_d + e_z


def mean_m(m):
    return np.asarray(m, dtype=np.float64).reshape(3, -1).mean(axis=1)
