"""Stored expected values are the oracle's, for the inputs the tests use (CPU only)."""
import importlib.util
import os

import numpy as np

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _module(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(HERE, "golden", name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_adjoint_fixture_matches_the_workload_inputs():
    gm = _module("make_adjoint_film_4096")
    gold = np.load(gm.OUT)
    w = workloads.adjoint_film()
    assert str(gold["digest"]) == gm.inputs_digest(w)
    assert int(gold["steps"]) == gm.STEPS == w.steps
    n = w.films[0].ncells
    assert gold["g_hext"].size == 3 * n and gold["g_ms"].size == n and gold["g_m0"].size == 3 * n
    for k in ("g_hext", "g_ms", "g_m0"):
        assert np.isfinite(gold[k]).all() and np.abs(gold[k]).max() > 0


def test_adjoint_fixture_loss_is_the_oracle_loss_of_its_target():
    """The stored loss is mean |m(T) - target|^2 of unit vectors: within [0, 4]; and the
    stored dL/dm_0 has the size of a gradient of such a loss (nonzero, finite)."""
    gm = _module("make_adjoint_film_4096")
    gold = np.load(gm.OUT)
    assert 0.0 < float(gold["loss"]) < 4.0
