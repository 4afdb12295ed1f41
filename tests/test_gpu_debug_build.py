"""The checked build (libgrace_debug.so, -DGRACE_DEBUG): the kernels record failed index and
shared-memory-extent checks in a workspace word instead of trapping, and every runtime
buffer is followed by a guard region.  Odd and edge shapes that take every launch path
(runtime-length x / y / z kernels, the fused and the split compile-time paths, the staged z
pass, a batch on the grouped and the persistent launch, Heun, the adjoint on both x passes) must leave the word clear and the guards intact, and give the
release library's results.

Each library runs in a subprocess of its own (GRACE_DEBUG selects which one the binding
loads)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import ctypes as C, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import workloads
from paper_1411_2565_gb300 import _lib, build
build.build(debug=_lib.DEBUG)
L = _lib.load()
from paper_1411_2565_gb300.grace import Grace, GraceBatch
res, arrays = {}, {}

def check(g, name):
    flags = C.c_uint(0)
    st = L.grace_debug_check(g.ctx, C.byref(flags))
    res[name] = [st, flags.value]

shapes = [(1, 1, 1), (3, 1, 1), (1, 7, 1), (9, 3, 6), (5, 5, 5), (33, 17, 3), (64, 16, 2),
          (40, 24, 8), (17, 1, 9), (20, 12, 1)]
for grid in shapes:
    f, m0 = workloads.small_film(grid, seed=7, Ku=1e4, alpha=0.2, hext=(1e4, -5e3, 2e3))
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, tuned=False)
    g.set_hext(f.hext)
    g.set_m(torch.from_numpy(m0.reshape(-1)).cuda())
    arrays["h%s" % (grid,)] = g.heff().cpu().numpy()
    g.step(5, 1e-14)
    arrays["m%s" % (grid,)] = g.get_m().cpu().numpy()
    check(g, "film%s" % (grid,))
    g.set_option(_lib.OPT_INTEGRATOR, 1)
    g.step(3, 1e-14)
    arrays["heun%s" % (grid,)] = g.get_m().cpu().numpy()
    check(g, "heun%s" % (grid,))
    g.close()
# the staged z pass (TMA copies of the spectrum columns) on a padded z length of 128
f, m0 = workloads.small_film((24, 20, 33), seed=8, Ku=1e4, alpha=0.2, hext=(1e4, -5e3, 2e3))
g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, options={_lib.OPT_TILE_Z: 4})
g.set_hext(f.hext)
g.set_m(torch.from_numpy(m0.reshape(-1)).cuda())
g.step(5, 1e-14)
arrays["staged_z"] = g.get_m().cpu().numpy()
check(g, "staged_z")
g.close()
w = workloads.ensemble(nfilms=8, seed=51)
mb = torch.from_numpy(np.concatenate([m.reshape(-1) for m in w.m0])).cuda()
for pers in (0, 1):
    b = GraceBatch(w.films, options={_lib.OPT_PERSISTENT: pers})
    b.set_m(mb)
    b.step(20, w.dt)
    b.sync()
    arrays["batch%d" % pers] = b.get_m().cpu().numpy()
    check(b, "batch%d" % pers)
    b.close()
for grid in [(24, 16, 2), (4, 6, 3)]:
    f, m0 = workloads.small_film(grid, seed=9, alpha=0.1)
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, tuned=False)
    g.set_m(torch.from_numpy(m0.reshape(-1)).cuda())
    n = 3 * f.ncells
    gm0 = g.backward(torch.linspace(-1e-3, 1e-3, n, device="cuda"), 13, 1e-14, 5,
                     torch.zeros(n, device="cuda"), torch.zeros(f.ncells, device="cuda"))
    arrays["adjoint%s" % (grid,)] = gm0.cpu().numpy()
    check(g, "adjoint%s" % (grid,))
    g.close()
np.savez(sys.argv[2], **arrays)
print(json.dumps(res))
"""


def _run(tmp_path, debug):
    out = str(tmp_path / ("debug.npz" if debug else "release.npz"))
    env = dict(os.environ, GRACE_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT, out], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_checked_build_is_clean_on_every_launch_path(tmp_path):
    res_d, arr_d = _run(tmp_path, True)
    for name, (st, flags) in res_d.items():
        assert st == 0 and flags == 0, (name, st, flags)
    res_r, arr_r = _run(tmp_path, False)
    for name, (st, _) in res_r.items():
        assert st == -7, name                  # GRACE_EUNSUPPORTED: the release build has no checks
    for k in arr_d.files:
        a, b = arr_d[k].astype(np.float64), arr_r[k].astype(np.float64)
        scale = max(1e-30, np.abs(b).max())
        assert np.abs(a - b).max() <= 1e-5 * scale, k
