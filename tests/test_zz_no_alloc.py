"""grace_energy_noalloc: the energy reduction for callers that cannot allocate device
memory (its FP64 partial sums live in a static device array inside the library).

Checks it through the C ABI against grace_energy, the workspace-based entry point, on
the same state and demag field, on two calls in a row (the second call must not be
affected by what the first left in the shared array), and the first call also against
the FP64 oracle's energies."""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
REL = 1e-9


def test_energy_noalloc_matches_workspace_energy_twice():
    libbuild.build()
    L = _lib.load()
    from paper_1411_2565_gb300.grace import Grace
    f, m0 = workloads.small_film((40, 24, 3), cell=(3e-9, 2.5e-9, 2e-9), seed=17, Ku=2e4,
                                 hext=(1.5e4, -1e4, 4e3))
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device="cuda:0")
    g.set_hext(f.hext)
    m = torch.from_numpy(m0.reshape(-1)).to("cuda:0")
    for call in range(2):
        if call == 1:                                  # a different state for the second call
            g.step(7, 1e-14)
            m = g.get_m()
        g.set_m(m)
        hd = g.heff(_lib.TERM_DEMAG)
        ref, ref_avg = g.energy()
        out = (C.c_double * 5)()
        avg = (C.c_double * 3)()
        stream = torch.cuda.current_stream().cuda_stream
        st = L.grace_energy_noalloc(_lib.ivec(f.grid), _lib.dvec(f.cell), f.Ms, f.A, f.Ku,
                                    _lib.dvec(f.hext), m.data_ptr(), hd.data_ptr(), stream, out, avg)
        assert st == 0, st
        names = ("exch", "anis", "demag", "zeeman", "total")
        scale = max(abs(ref[k]) for k in names)
        for k, name in enumerate(names):
            assert abs(out[k] - ref[name]) <= REL * scale, (call, name, out[k], ref[name])
        assert np.allclose(list(avg), ref_avg, rtol=0, atol=1e-12)
        if call == 0:
            # and directly against the FP64 oracle's Eq. 1 energies of the same state
            from oracle import llg
            p = llg.Params(f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, f.hext)
            oref = llg.energies(m0, p)
            oscale = max(abs(v) for v in oref[:4])
            for k in range(5):
                assert abs(out[k] - oref[k]) <= 2e-6 * oscale + 1e-6 * abs(oref[k]), (k, out[k], oref[k])


def test_energy_noalloc_rejects_oversized_grid():
    libbuild.build()
    L = _lib.load()
    st = L.grace_energy_noalloc(_lib.ivec([2048, 2048, 8]), _lib.dvec([1e-9] * 3), 8e5, 1e-11, 0.0,
                                _lib.dvec([0, 0, 0]), C.c_void_p(16), C.c_void_p(16), None,
                                None, None)
    assert st == -7        # GRACE_EUNSUPPORTED: more cells than the static scratch covers
