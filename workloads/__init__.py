"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no micromagnetic arithmetic: it only draws random numbers and
describes the workload shapes.  Both the CUDA path and the FP64 oracle receive
the *same* FP32 arrays produced here, so a parity comparison never depends on
which side generated its input.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output i of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.  It is counter based, so any
element can be regenerated independently and the stream is identical on x86
and Arm hosts.

Workloads (Sec. 4 of the paper shapes them: N^3 cubes in Table 1 and the
500x125x3 nm muMAG #4 film; the concrete sizes below are the synthetic
stand-ins this project measures):

* ``film_small``  128x32x1 film, 3.90625x3.90625x3 nm cells, S-state start.
* ``film_large``  1024x256x4 film, 2 nm cubic cells, random start, 25 mT field.
* ``block``       256x256x64 block, 3 nm cells, random start.
* ``ensemble``    256 independent films of four sizes with random materials.
* ``adjoint``     256x64x2 film, 4x4x3 nm cells, per-cell Ms, smooth target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

MU0 = 4e-7 * math.pi          # vacuum permeability, SI (exact pre-2019 value)
GAMMA0 = 2.211e5              # gyromagnetic ratio times mu0, m/(A s)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform of consecutive uniform pairs."""
    u = uniform(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]                       # (0, 1]: log is finite
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def random_unit_m(shape_zyx: Tuple[int, int, int], seed: int) -> np.ndarray:
    """Random unit vectors (isotropic): normalised Gaussian 3-vectors, FP32, layout [3][nz][ny][nx]."""
    n = int(np.prod(shape_zyx))
    g = gaussian(seed, 3 * n).reshape(3, *shape_zyx)
    g /= np.sqrt((g * g).sum(axis=0, keepdims=True))
    return np.ascontiguousarray(g.astype(np.float32))


def s_state_m(shape_zyx: Tuple[int, int, int], seed: int, noise: float = 0.01) -> np.ndarray:
    """Seeded S-like start: m = (cos t, sin t, 0), t(i) = (pi/6)[e^{-(i+1/2)/w} + e^{-(nx-i-1/2)/w}],
    w = nx/8, plus uniform +-noise per component, normalised; FP32 [3][nz][ny][nx]."""
    nz, ny, nx = shape_zyx
    i = np.arange(nx, dtype=np.float64) + 0.5
    w = nx / 8.0
    t = (math.pi / 6.0) * (np.exp(-i / w) + np.exp(-(nx - i) / w))
    m = np.zeros((3, nz, ny, nx))
    m[0] = np.cos(t)[None, None, :]
    m[1] = np.sin(t)[None, None, :]
    m += noise * (2.0 * uniform(seed, m.size).reshape(m.shape) - 1.0)
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return np.ascontiguousarray(m.astype(np.float32))


def near_saturated_m(shape_zyx: Tuple[int, int, int], direction, seed: int, noise: float = 0.02) -> np.ndarray:
    """Uniform m along `direction` plus uniform +-noise per component, normalised; FP32
    [3][nz][ny][nx] (the near-saturated start of the standard-problem-4 relaxation)."""
    d = np.asarray(direction, dtype=np.float64)
    m = np.broadcast_to((d / np.linalg.norm(d))[:, None, None, None], (3,) + tuple(shape_zyx)).copy()
    m += noise * (2.0 * uniform(seed, m.size).reshape(m.shape) - 1.0)
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return np.ascontiguousarray(m.astype(np.float32))


def smooth_target(shape_zyx: Tuple[int, int, int], seed: int) -> np.ndarray:
    """Smooth unit target field normalise(cos(2 pi x/Lx + p1), sin(2 pi y/Ly + p2), 0.3 cos(2 pi (x+y)/Lx + p3))."""
    nz, ny, nx = shape_zyx
    p = 2.0 * math.pi * uniform(seed, 3)
    x = (np.arange(nx) + 0.5)[None, None, :] / nx
    y = (np.arange(ny) + 0.5)[None, :, None] / ny
    t = np.zeros((3, nz, ny, nx))
    t[0] = np.cos(2 * math.pi * x + p[0])
    t[1] = np.sin(2 * math.pi * y + p[1])
    t[2] = 0.3 * np.cos(2 * math.pi * (x + y * ny / nx) + p[2])
    t /= np.sqrt((t * t).sum(axis=0, keepdims=True))
    return np.ascontiguousarray(t.astype(np.float32))


@dataclass
class Film:
    """One rectangular film: grid (nx, ny, nz), cell (m), material, applied field (A/m)."""
    grid: Tuple[int, int, int]
    cell: Tuple[float, float, float]
    Ms: float
    A: float
    Ku: float
    alpha: float
    gamma0: float = GAMMA0
    hext: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    @property
    def ncells(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def shape_zyx(self) -> Tuple[int, int, int]:
        return (self.grid[2], self.grid[1], self.grid[0])


@dataclass
class Workload:
    name: str
    films: List[Film]
    steps: int
    dt: float
    m0: List[np.ndarray] = field(default_factory=list)
    note: str = ""
    ms_field: Optional[np.ndarray] = None
    target: Optional[np.ndarray] = None


def padded(n: int) -> int:
    """Smallest power of two >= 2n-1 (1 for n == 1): the zero-padded FFT length."""
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def _field_from_mT(b_mT: float, angle_deg: float) -> Tuple[float, float, float]:
    h = b_mT * 1e-3 / MU0
    a = math.radians(angle_deg)
    return (h * math.cos(a), h * math.sin(a), 0.0)


def film_small() -> Workload:
    f = Film((128, 32, 1), (3.90625e-9, 3.90625e-9, 3e-9), Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.5)
    return Workload("film_small 128x32x1", [f], steps=500, dt=1e-14,
                    m0=[s_state_m(f.shape_zyx, seed=1)],
                    note="S-state + 0.01 noise (seed 1)")


def film_large() -> Workload:
    f = Film((1024, 256, 4), (2e-9, 2e-9, 2e-9), Ms=8.6e5, A=1.3e-11, Ku=5e2, alpha=0.02,
             hext=_field_from_mT(25.0, 170.0))
    return Workload("film_large 1024x256x4", [f], steps=10000, dt=5e-15,
                    m0=[random_unit_m(f.shape_zyx, seed=2)],
                    note="random unit m (seed 2), 25 mT at 170 deg")


def block() -> Workload:
    f = Film((256, 256, 64), (3e-9, 3e-9, 3e-9), Ms=1.0e6, A=1.5e-11, Ku=1e4, alpha=0.1)
    return Workload("block 256x256x64", [f], steps=1000, dt=1e-14,
                    m0=[random_unit_m(f.shape_zyx, seed=3)], note="random unit m (seed 3)")


ENSEMBLE_SIZES = [(64, 16, 1), (128, 32, 1), (256, 64, 2), (200, 50, 1)]


def ensemble(nfilms: int = 256, seed: int = 4) -> Workload:
    """Random films; draws in the order size, Ms, alpha, |B|, angle (one stream per quantity), then m."""
    u_size = uniform(seed, nfilms, 0)
    u_ms = uniform(seed + 1000, nfilms)
    u_al = uniform(seed + 2000, nfilms)
    u_b = uniform(seed + 3000, nfilms)
    u_an = uniform(seed + 4000, nfilms)
    films, m0 = [], []
    for k in range(nfilms):
        g = ENSEMBLE_SIZES[min(int(u_size[k] * 4), 3)]
        b = 50.0 * u_b[k]
        ang = 360.0 * u_an[k]
        f = Film(g, (3.90625e-9, 3.90625e-9, 3e-9), Ms=4e5 + 8e5 * u_ms[k], A=1.3e-11, Ku=0.0,
                 alpha=0.01 + 0.49 * u_al[k], hext=_field_from_mT(b, ang))
        films.append(f)
        m0.append(random_unit_m(f.shape_zyx, seed=seed * 100000 + k))
    return Workload(f"ensemble {nfilms} films", films, steps=2000, dt=1e-14, m0=m0,
                    note="sizes from {64x16x1,128x32x1,256x64x2,200x50x1}")


def adjoint_film() -> Workload:
    f = Film((256, 64, 2), (4e-9, 4e-9, 3e-9), Ms=8.0e5, A=1.3e-11, Ku=0.0, alpha=0.1)
    w = Workload("adjoint 256x64x2", [f], steps=4096, dt=1e-14,
                 m0=[random_unit_m(f.shape_zyx, seed=5)], note="per-cell Ms, target seed 6")
    w.ms_field = np.full(f.shape_zyx, f.Ms, dtype=np.float32)
    w.target = smooth_target(f.shape_zyx, seed=6)
    return w


def small_film(grid, cell=(3e-9, 3e-9, 3e-9), seed=11, Ms=8e5, A=1.3e-11, Ku=0.0, alpha=0.1,
               hext=(0.0, 0.0, 0.0)) -> Tuple[Film, np.ndarray]:
    """A small random-start film for parity and edge-case tests."""
    f = Film(tuple(grid), tuple(cell), Ms=Ms, A=A, Ku=Ku, alpha=alpha, hext=tuple(hext))
    return f, random_unit_m(f.shape_zyx, seed)
