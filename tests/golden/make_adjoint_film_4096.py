"""Write ``adjoint_film_4096.npz``: the FP64 oracle's gradients on the adjoint workload.

The adjoint film is 256x64x2 cells of 4x4x3 nm with a per-cell Ms (seed 5 start, seed 6
target; ``workloads.adjoint_film``) and a zero per-cell applied field.  Through 4,096
explicit Euler steps at dt = 1e-14 s (Eq. 3, renormalised) the oracle's exact discrete
adjoint gives, for the loss L = mean |m(T) - m_target|^2:

  dL/dH_ext per cell (3 N), dL/dMs per cell (N), dL/dm_0 (3 N), and L itself.

Only ``oracle/`` and the seeded input generators are called; nothing here comes from
the CUDA path.  The arrays are stored in FP32 (their rounding, ~1e-7 relative, is far
below the 1e-3 relative-L2 bar the GPU gradients are held to) with a digest of the
inputs, so a test can tell when the fixture no longer matches the workload.

    python tests/golden/make_adjoint_film_4096.py        # ~10 minutes, ~3.3 GB of host memory
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

STEPS = 4096
OUT = os.path.join(HERE, "adjoint_film_4096.npz")


def inputs_digest(w) -> str:
    """sha256 over the workload's FP32 inputs, its step and its material constants."""
    f = w.films[0]
    h = hashlib.sha256()
    for a in (w.m0[0], w.ms_field, w.target):
        h.update(np.ascontiguousarray(a, dtype=np.float32).tobytes())
    h.update(repr((f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, w.dt, STEPS)).encode())
    return h.hexdigest()


def main():
    import workloads
    from oracle import adjoint as oadj
    from oracle import llg
    w = workloads.adjoint_film()
    f, m0 = w.films[0], w.m0[0]
    h = np.zeros((3,) + f.shape_zyx)
    p = llg.Params(f.cell, w.ms_field.astype(np.float64), f.A, f.Ku, f.alpha, f.gamma0, h)
    t0 = time.time()
    loss, g_m0, g_h, g_ms = oadj.gradients(m0, p, w.dt, STEPS, w.target)
    np.savez_compressed(OUT, loss=np.float64(loss), g_hext=g_h.astype(np.float32),
                        g_ms=g_ms.astype(np.float32), g_m0=g_m0.astype(np.float32),
                        steps=np.int64(STEPS), digest=np.array(inputs_digest(w)))
    print(f"wrote {OUT}: loss {loss:.9e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
