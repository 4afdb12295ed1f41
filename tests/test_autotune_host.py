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
    assert at.best(films) == {int(k): v for k, v in mine.items()}
    with open(at.CACHE) as fh:
        assert json.load(fh)[key]["options"] == mine
