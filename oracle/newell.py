"""Cell-averaged demagnetisation tensor between two equal rectangular cells, FP64.

The paper computes the demag field as the discrete convolution of M with "the
demagnetization tensor" evaluated by FFT with zero padding (Sec. 3, citing [3],
Newell, Williams & Dunlop, J. Geophys. Res. 98, 9551 (1993)).  The tensor itself is
not printed in the paper; this module states the reading used throughout:

N_ab(r) for an offset r between the centres of two cells of size (dx, dy, dz) is the
field at an observer cell, averaged over that cell, produced by a uniformly magnetised
source cell with unit magnetisation along b, with H = -N M.

* Near field (Chebyshev distance in cells <= ``R_SWITCH``): Newell's closed form, a
  27-point second difference (weights -1, 2, -1 per axis) of the functions f (diagonal
  components) and g (off-diagonal components), divided by 4 pi dx dy dz.
* Far field: the point-dipole tensor plus its second-order cell-shape correction.  The
  cell-averaged tensor is the dipole kernel averaged over the difference u of two
  uniform points in the two cells; each component of u has variance d^2/6, so to second
  order N(r) = D(r) + (1/12) sum_d dd^2 d^2D/dr_d^2 (the term vanishes for cubic cells
  because D is harmonic).  FP64 Newell loses digits to cancellation at large distance
  (~1e-7 relative at 24 cells), while this asymptote's error falls as (cell/r)^4 (~1e-7
  at 24 cells); 24 cells is the crossover.
"""
from __future__ import annotations

import numpy as np

R_SWITCH = 24          # Chebyshev radius (cells) of the Newell region


def _safe_div(a, b):
    """a / b, with 0 where b == 0 (those terms carry a zero prefactor)."""
    b_ok = np.where(b == 0.0, 1.0, b)
    return np.where(b == 0.0, 0.0, a / b_ok)


def newell_f(x, y, z):
    """Newell's f(x, y, z) (even in each argument); terms with a zero denominator are dropped."""
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = 0.5 * y * (z2 - x2) * np.arcsinh(_safe_div(y, np.sqrt(x2 + z2)))
    t = t + 0.5 * z * (y2 - x2) * np.arcsinh(_safe_div(z, np.sqrt(x2 + y2)))
    t = t - x * y * z * np.arctan(_safe_div(y * z, x * R))
    t = t + (2.0 * x2 - y2 - z2) * R / 6.0
    return t


def newell_g(x, y, z):
    """Newell's g(x, y, z): sgn(x) sgn(y) times the expression evaluated on |x|, |y|, |z|."""
    s = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = x * y * z * np.arcsinh(_safe_div(z, np.sqrt(x2 + y2)))
    t = t + y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(_safe_div(x, np.sqrt(y2 + z2)))
    t = t + x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(_safe_div(y, np.sqrt(x2 + z2)))
    t = t - z2 * z / 6.0 * np.arctan(_safe_div(x * y, z * R))
    t = t - 0.5 * z * y2 * np.arctan(_safe_div(x * z, y * R))
    t = t - 0.5 * z * x2 * np.arctan(_safe_div(y * z, x * R))
    t = t - x * y * R / 3.0
    return s * t


_W = {-1: -1.0, 0: 2.0, 1: -1.0}


def _second_difference(fun, X, Y, Z, dx, dy, dz):
    acc = 0.0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                acc = acc + _W[i] * _W[j] * _W[k] * fun(X + i * dx, Y + j * dy, Z + k * dz)
    return acc / (4.0 * np.pi * dx * dy * dz)


def newell_tensor(X, Y, Z, dx, dy, dz):
    """(Nxx, Nyy, Nzz, Nxy, Nxz, Nyz) at centre offset (X, Y, Z) metres, Newell's closed form."""
    X, Y, Z = (np.asarray(v, dtype=np.float64) for v in (X, Y, Z))
    nxx = _second_difference(newell_f, X, Y, Z, dx, dy, dz)
    nyy = _second_difference(newell_f, Y, X, Z, dy, dx, dz)
    nzz = _second_difference(newell_f, Z, Y, X, dz, dy, dx)
    nxy = _second_difference(newell_g, X, Y, Z, dx, dy, dz)
    nxz = _second_difference(newell_g, X, Z, Y, dx, dz, dy)
    nyz = _second_difference(newell_g, Y, Z, X, dy, dz, dx)
    return nxx, nyy, nzz, nxy, nxz, nyz


_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def asymptotic_tensor(X, Y, Z, dx, dy, dz):
    """Point dipole V (delta r^2 - 3 r r)/(4 pi r^5) plus the second-order cell-average term.

    With phi = 1/r, D_ab = -(V/4pi) d_a d_b phi and the correction is
    -(V/4pi)(1/12) sum_d dd^2 d_a d_b d_d d_d phi, using the fourth derivative of 1/r:
    105 x_a x_b x_d^2/r^9 - 15(delta_ab x_d^2 + 2 delta_ad x_b x_d + 2 delta_bd x_a x_d
    + x_a x_b)/r^7 + 3(delta_ab + 2 delta_ad delta_bd)/r^5.
    """
    x = [np.asarray(v, dtype=np.float64) for v in (X, Y, Z)]
    h2 = (dx * dx, dy * dy, dz * dz)
    r2 = x[0] ** 2 + x[1] ** 2 + x[2] ** 2
    r = np.sqrt(r2)
    r5, r7, r9 = r2 * r2 * r, r2 ** 3 * r, r2 ** 4 * r
    pref = dx * dy * dz / (4.0 * np.pi)
    out = []
    for a, b in _PAIRS:
        dab = 1.0 if a == b else 0.0
        dip = pref * (dab * r2 - 3.0 * x[a] * x[b]) / r5
        corr = 0.0
        for d in range(3):
            dad = 1.0 if a == d else 0.0
            dbd = 1.0 if b == d else 0.0
            t = (105.0 * x[a] * x[b] * x[d] ** 2 / r9
                 - 15.0 * (dab * x[d] ** 2 + 2.0 * dad * x[b] * x[d] + 2.0 * dbd * x[a] * x[d]
                           + x[a] * x[b]) / r7
                 + 3.0 * (dab + 2.0 * dad * dbd) / r5)
            corr = corr + h2[d] * t
        out.append(dip - pref * corr / 12.0)
    return tuple(out)


def demag_tensor(ix, iy, iz, cell, r_switch: int = R_SWITCH):
    """Tensor at integer cell offsets (ix, iy, iz) (arrays, broadcast), cell = (dx, dy, dz).

    Returns the six components (xx, yy, zz, xy, xz, yz) as FP64 arrays.
    """
    dx, dy, dz = (float(c) for c in cell)
    ix, iy, iz = np.broadcast_arrays(*(np.asarray(v, dtype=np.int64) for v in (ix, iy, iz)))
    cheb = np.maximum(np.maximum(np.abs(ix), np.abs(iy)), np.abs(iz))
    near = cheb <= r_switch
    out = [np.zeros(ix.shape) for _ in range(6)]
    if near.any():
        vals = newell_tensor(ix[near] * dx, iy[near] * dy, iz[near] * dz, dx, dy, dz)
        for o, v in zip(out, vals):
            o[near] = v
    far = ~near
    if far.any():
        vals = asymptotic_tensor(ix[far] * dx, iy[far] * dy, iz[far] * dz, dx, dy, dz)
        for o, v in zip(out, vals):
            o[far] = v
    return tuple(out)
