"""The GPU demag convolution against closed forms of a discrete convolution (GB300, through
the C ABI; Sec. 3: H_demag as the zero-padded FFT convolution of M with the tensor).

* Impulse: with one magnetised cell (m = e at r_0, zero elsewhere) the convolution returns
  the tensor itself, H(r_i) = -Ms N(r_i - r_0) e at every cell i, for N from the oracle's
  FP64 tensor; this pins the forward transforms, the tensor product with its parities,
  the inverse transforms and the crop, on the fused, split and runtime-length paths,
  with impulses at a corner, an edge and inside.
* Linearity: H(m1 + m2) = H(m1) + H(m2).

Tolerance: max |dH| / Ms <= 1e-5, as for every field evaluation.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle.newell import demag_tensor
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
TOL_H = 1e-5
DEV = "cuda:0"
MS = 8e5
CELL = (3.5e-9, 2.5e-9, 3e-9)


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return _lib.load()


def demag_field(grid, m):
    from paper_1411_2565_gb300.grace import Grace
    with Grace(grid, CELL, MS, 1.3e-11, 0.0, 0.1, device=DEV) as g:
        g.set_m(torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32).reshape(-1)).to(DEV))
        return g.heff(1).cpu().numpy().reshape(m.shape).astype(np.float64)


def impulse_reference(grid, r0, e):
    nx, ny, nz = grid
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xx, yy, zz, xy, xz, yz = demag_tensor(xs - r0[0], ys - r0[1], zs - r0[2], CELL)
    return -MS * np.stack([xx * e[0] + xy * e[1] + xz * e[2],
                           xy * e[0] + yy * e[1] + yz * e[2],
                           xz * e[0] + yz * e[1] + zz * e[2]])


GRIDS = [(16, 8, 2), (40, 20, 4), (17, 5, 3), (9, 3, 6), (12, 6, 9), (5, 40, 1), (33, 9, 5), (64, 3, 2)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("where", ["corner", "edge", "inside"])
def test_impulse_returns_the_tensor(grid, where):
    nx, ny, nz = grid
    r0 = {"corner": (0, 0, 0), "edge": (nx - 1, ny // 2, 0),
          "inside": (nx // 2, ny // 3, nz // 2)}[where]
    e = np.array([0.3, -0.5, 0.8], dtype=np.float32)
    e /= np.linalg.norm(e)
    m = np.zeros((3, nz, ny, nx), dtype=np.float32)
    m[:, r0[2], r0[1], r0[0]] = e
    h = demag_field(grid, m)
    ref = impulse_reference(grid, r0, e.astype(np.float64))
    err = np.abs(h - ref).max() / MS
    assert err <= TOL_H, f"grid {grid}, impulse at {r0}: {err:.3e}"


@pytest.mark.parametrize("grid", [(24, 12, 2), (12, 6, 9), (17, 5, 3)])
def test_convolution_is_linear(grid):
    nx, ny, nz = grid
    m1 = workloads.random_unit_m((nz, ny, nx), seed=71)
    m2 = workloads.random_unit_m((nz, ny, nx), seed=72)
    m3 = (m1 + m2).astype(np.float32)
    h1, h2, h3 = demag_field(grid, m1), demag_field(grid, m2), demag_field(grid, m3)
    err = np.abs(h3 - (h1 + h2)).max() / MS
    assert err <= TOL_H, f"grid {grid}: {err:.3e}"
