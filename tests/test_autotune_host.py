"""Host logic of the autotuner (CPU only): cache keys, the shipped GB300 schedule table and
the precedence of a local cache over it.  The device name is faked; nothing is timed."""
import json

import pytest
import torch

import workloads
from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import autotune as at

WORKLOADS = ("film_large", "block", "film_small", "ensemble", "adjoint_film")


@pytest.fixture
def gb300(monkeypatch, tmp_path):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "NVIDIA GB300")
    monkeypatch.setattr(at, "CACHE", str(tmp_path / "cache.json"))
    return tmp_path


@pytest.mark.parametrize("name", WORKLOADS)
def test_shipped_table_covers_the_benchmark_shapes(gb300, name):
    films = getattr(workloads, name)().films
    opts = at.best(films)
    assert set(opts) == set(at.CANDIDATES)
    for k, v in opts.items():
        assert v in at.CANDIDATES[k]


def test_key_ignores_film_order_and_depends_on_shapes_and_device(gb300, monkeypatch):
    films = workloads.ensemble().films
    dev = torch.device("cuda")
    k = at._key(films, dev)
    assert at._key(list(reversed(films)), dev) == k
    assert at._key(films[:-1], dev) != k
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "another GPU")
    assert at._key(films, dev) != k
    assert at.best(films) == {}                       # nothing shipped for another device


def test_local_cache_takes_precedence(gb300):
    films = workloads.film_large().films
    key = at._key(films, torch.device("cuda"))
    mine = {str(_lib.OPT_TILE_X): 0, str(_lib.OPT_TILE_YZ): 1, str(_lib.OPT_GRAPH_STEPS): 8,
            str(_lib.OPT_PDL): 0}
    at._store({key: {"options": mine, "ms_per_step": 1.0, "films": 1, "tried": 1}})
    want = dict(at.DEFAULTS)
    want.update({int(k): v for k, v in mine.items()})
    assert at.best(films) == want              # options the entry predates keep their defaults
    with open(at.CACHE) as fh:
        assert json.load(fh)[key]["options"] == mine


def test_only_options_that_can_matter_are_searched():
    film = workloads.film_large().films
    block = workloads.block().films
    ens = workloads.ensemble().films
    assert at.relevant(film)[_lib.OPT_TILE_YZ] and not at.relevant(film)[_lib.OPT_TILE_Z]
    assert at.relevant(block)[_lib.OPT_TILE_Z] and not at.relevant(block)[_lib.OPT_TILE_YZ]
    assert at.relevant(ens)[_lib.OPT_SIDE_STREAMS] and not at.relevant(film)[_lib.OPT_SIDE_STREAMS]
    for k, v in at.DEFAULTS.items():
        assert v in at.CANDIDATES[k]


def test_binding_applies_the_tuned_schedule_unless_told_not_to(gb300, monkeypatch):
    from paper_1411_2565_gb300 import grace
    films = workloads.block().films
    f = films[0]
    shape = grace._Shape(f.grid, f.cell)
    assert at._key([shape], torch.device("cuda")) == at._key(films, torch.device("cuda"))
    assert grace._tuned([shape], "cuda", None, True) == at.best(films)
    assert grace._tuned([shape], "cuda", None, False) == {}
    mine = {_lib.OPT_TILE_X: 1}
    assert grace._tuned([shape], "cuda", mine, True) == mine
