"""Demagnetising field H_d = -N * M on a regular grid, FP64 (paper Sec. 1 and Sec. 3).

Two independent evaluations of the same discrete convolution:

* ``demag_direct``  the O(N^2) sum H_i = -sum_j N(r_i - r_j) M_j over every source cell
  (the brute-force method of Sec. 1), for tiny grids and for sampled cells of large ones.
* ``demag_fft``     the zero-padded FFT convolution of Sec. 3: each axis padded to
  P_d = the smallest power of two >= 2 n_d - 1 (P_d = 1 when n_d = 1), the tensor placed
  with offset -k at index P_d - k, numpy's FFT as the transform primitive.  Any
  P_d >= 2 n_d - 1 gives the same linear (non-periodic) convolution.

M = Ms m, with Ms a scalar or a per-cell array [nz][ny][nx].
"""
from __future__ import annotations

import numpy as np

from .newell import R_SWITCH, demag_tensor


def padded_length(n: int) -> int:
    """Smallest power of two >= 2n - 1 (1 for n == 1)."""
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def offset_tensor(grid, cell, r_switch: int = R_SWITCH):
    """Six tensor components on every offset in [-(n-1), n-1]^3, shaped (2nz-1, 2ny-1, 2nx-1).

    Index (kz, ky, kx) holds offset (kx - (nx-1), ky - (ny-1), kz - (nz-1)).
    """
    nx, ny, nz = grid
    ox = np.arange(-(nx - 1), nx)[None, None, :]
    oy = np.arange(-(ny - 1), ny)[None, :, None]
    oz = np.arange(-(nz - 1), nz)[:, None, None]
    return demag_tensor(ox, oy, oz, cell, r_switch)


def _magnetisation(m, Ms):
    return np.asarray(m, dtype=np.float64) * np.asarray(Ms, dtype=np.float64)


def demag_direct(m, Ms, cell, r_switch: int = R_SWITCH):
    """H_i = -sum_j N(r_i - r_j) M_j by explicit summation over all pairs (O(N^2))."""
    M = _magnetisation(m, Ms)
    _, nz, ny, nx = M.shape
    N = offset_tensor((nx, ny, nz), cell, r_switch)
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4,
            (1, 2): 5, (2, 1): 5}
    H = np.zeros_like(M)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                # offsets r_i - r_j for all sources j: index (i - j) + (n - 1)
                win = (slice(z + nz - 1, z - 1 if z > 0 else None, -1),
                       slice(y + ny - 1, y - 1 if y > 0 else None, -1),
                       slice(x + nx - 1, x - 1 if x > 0 else None, -1))
                for a in range(3):
                    s = 0.0
                    for b in range(3):
                        s += np.sum(N[comp[(a, b)]][win] * M[b])
                    H[a, z, y, x] = -s
    return H


def demag_at(cells, m, Ms, cell, r_switch: int = R_SWITCH):
    """Direct sum at selected observer cells ``cells`` = list of (x, y, z); returns (len, 3)."""
    M = _magnetisation(m, Ms)
    _, nz, ny, nx = M.shape
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((len(cells), 3))
    for k, (x, y, z) in enumerate(cells):
        nxx, nyy, nzz, nxy, nxz, nyz = demag_tensor(x - xs, y - ys, z - zs, cell, r_switch)
        Mx, My, Mz = M[0], M[1], M[2]
        out[k, 0] = -np.sum(nxx * Mx + nxy * My + nxz * Mz)
        out[k, 1] = -np.sum(nxy * Mx + nyy * My + nyz * Mz)
        out[k, 2] = -np.sum(nxz * Mx + nyz * My + nzz * Mz)
    return out


def padded_tensor_spectrum(grid, cell, r_switch: int = R_SWITCH):
    """rfftn of the six tensor components placed on the padded grid (wrap: -k -> P - k)."""
    nx, ny, nz = grid
    P = (padded_length(nz), padded_length(ny), padded_length(nx))
    comps = offset_tensor(grid, cell, r_switch)
    iz = np.arange(-(nz - 1), nz) % P[0]
    iy = np.arange(-(ny - 1), ny) % P[1]
    ix = np.arange(-(nx - 1), nx) % P[2]
    spec = []
    for c in comps:
        g = np.zeros(P)
        g[np.ix_(iz, iy, ix)] = c
        spec.append(np.fft.rfftn(g))
    return P, spec


def demag_fft(m, Ms, cell, spectrum=None, r_switch: int = R_SWITCH):
    """Zero-padded FFT convolution H = -IFFT(N^ . FFT(M)), cropped to the body."""
    M = _magnetisation(m, Ms)
    _, nz, ny, nx = M.shape
    if spectrum is None:
        spectrum = padded_tensor_spectrum((nx, ny, nz), cell, r_switch)
    P, (sxx, syy, szz, sxy, sxz, syz) = spectrum
    Mh = [np.fft.rfftn(M[c], s=P, axes=(0, 1, 2)) for c in range(3)]
    Hh = (sxx * Mh[0] + sxy * Mh[1] + sxz * Mh[2],
          sxy * Mh[0] + syy * Mh[1] + syz * Mh[2],
          sxz * Mh[0] + syz * Mh[1] + szz * Mh[2])
    return np.stack([-np.fft.irfftn(h, s=P, axes=(0, 1, 2))[:nz, :ny, :nx] for h in Hh])
