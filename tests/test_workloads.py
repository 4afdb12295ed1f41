"""The seeded input generators shared by the oracle and the CUDA path (CPU only)."""
import numpy as np

import workloads


def test_splitmix64_matches_its_published_sequence():
    # seed 0: the first outputs of the reference splitmix64 generator
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in workloads.splitmix64(0, 3)] == ref


def test_streams_are_counter_based():
    full = workloads.splitmix64(12345, 20)
    assert np.array_equal(workloads.splitmix64(12345, 7, offset=9), full[9:16])
    assert not np.array_equal(workloads.splitmix64(12346, 20), full)


def test_uniform_and_gaussian_moments():
    u = workloads.uniform(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1 / 12) < 5e-3
    g = workloads.gaussian(8, 200000)
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1.0) < 1e-2


def test_initial_states_are_unit_vectors_in_fp32():
    for m in (workloads.random_unit_m((2, 5, 7), 3), workloads.s_state_m((1, 8, 32), 1),
              workloads.near_saturated_m((1, 4, 16), (1, 1, 1), 10)):
        assert m.dtype == np.float32 and m.shape[0] == 3
        n = np.sqrt((m.astype(np.float64) ** 2).sum(0))
        assert np.abs(n - 1).max() < 1e-6


def test_workloads_have_the_stated_shapes():
    assert workloads.film_large().films[0].grid == (1024, 256, 4)
    assert workloads.block().films[0].grid == (256, 256, 64)
    w = workloads.ensemble()
    assert len(w.films) == 256 and {f.grid for f in w.films} <= set(workloads.ENSEMBLE_SIZES)
    assert all(4e5 <= f.Ms <= 1.2e6 and 0.01 <= f.alpha <= 0.5 for f in w.films)
