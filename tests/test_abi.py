"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/grace.h declares, and validates arguments and call order on the host."""
import ctypes as C
import os
import re

import pytest

from paper_1411_2565_gb300 import _lib
from paper_1411_2565_gb300 import build as libbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "grace.h")
EINVAL, EWORKSPACE, ESTATE = -1, -2, -5


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\s*\*)\s*(grace_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def _create(lib, grid=(16, 8, 2), cell=(3e-9, 3e-9, 3e-9), Ms=8e5, A=1.3e-11, Ku=0.0, alpha=0.1,
            g0=2.211e5):
    ctx = C.c_void_p()
    st = lib.grace_create(C.byref(ctx), _lib.ivec(grid), _lib.dvec(cell), Ms, A, Ku, alpha, g0)
    return st, ctx


@pytest.mark.parametrize("kw", [dict(grid=(0, 8, 2)), dict(grid=(16, 8, 4097)), dict(grid=(2049, 1, 1)),
                                dict(grid=(1, 2049, 1)), dict(grid=(1, 1, 2049)), dict(grid=(-1, 1, 1)),
                                dict(grid=(2048, 2048, 2048)), dict(grid=(1024, 1024, 683)), dict(cell=(0, 1e-9, 1e-9)),
                                dict(Ms=0.0), dict(Ms=-1.0), dict(A=-1e-11), dict(alpha=-0.1),
                                dict(g0=0.0), dict(Ms=float("nan"))])
def test_create_rejects_invalid_arguments(lib, kw):
    st, ctx = _create(lib, **kw)
    assert st == EINVAL
    assert not ctx.value


def test_largest_axis_is_accepted(lib):
    """Each axis up to 2048 cells, and films up to 715,827,882 cells (3 N within 32-bit
    indexing) are planned."""
    for grid in [(2048, 1, 1), (1, 2048, 1), (1, 1, 2048), (1024, 1024, 682)]:
        st, ctx = _create(lib, grid=grid)
        assert st == 0
        assert lib.grace_destroy(ctx) == 0


def test_create_plans_workspace_and_counts_cells(lib):
    st, ctx = _create(lib, grid=(1024, 256, 4), cell=(2e-9,) * 3)
    assert st == 0
    n = C.c_longlong()
    assert lib.grace_ncells(ctx, C.byref(n)) == 0 and n.value == 1024 * 256 * 4
    sz = C.c_size_t()
    assert lib.grace_workspace_size(ctx, C.byref(sz)) == 0
    N = n.value
    Kx, Ky = 1025, 257
    tensor = Kx * (6 * 4 - 2) * Ky * 4
    spectrum = 3 * 4 * Kx * 256 * 8
    state = 3 * (3 * N * 4)
    assert sz.value >= tensor + spectrum + state
    assert sz.value < 2 * (tensor + spectrum + state) + (1 << 20)
    lib.grace_destroy(ctx)


def test_workspace_of_the_largest_film_does_not_wrap(lib):
    """1024 x 1024 x 682 cells (the largest cell count a film may have along these axes):
    the workspace is planned in 64-bit sizes (spectrum with Py rows, FFT-z tensor, four
    state-sized arrays)."""
    st, ctx = _create(lib, grid=(1024, 1024, 682), cell=(2e-9,) * 3)
    assert st == 0
    sz = C.c_size_t()
    assert lib.grace_workspace_size(ctx, C.byref(sz)) == 0
    N = 1024 * 1024 * 682
    Kx, Py, Ky, Kz = 1025, 2048, 1025, 1025
    spectrum = 3 * 682 * Kx * Py * 8
    tensor = Kx * Ky * (6 * Kz) * 4
    state = 4 * 3 * N * 4
    assert sz.value >= spectrum + tensor + state > 2 ** 36
    assert sz.value < 2 * (spectrum + tensor + state)
    lib.grace_destroy(ctx)


def test_call_order_and_workspace_checks(lib):
    st, ctx = _create(lib)
    assert st == 0
    out = C.c_void_p(0x1000)
    assert lib.grace_step(ctx, 1, 1e-14) == ESTATE
    assert lib.grace_heff(ctx, out, 15) == ESTATE
    assert lib.grace_set_m(ctx, out) == ESTATE
    assert b"bind" in lib.grace_last_error(ctx)
    sz = C.c_size_t()
    lib.grace_workspace_size(ctx, C.byref(sz))
    assert lib.grace_bind(ctx, None, sz.value, None) == EINVAL
    assert lib.grace_bind(ctx, C.c_void_p(0x10010), sz.value, None) == EWORKSPACE
    assert lib.grace_bind(ctx, C.c_void_p(0x10000), sz.value - 1, None) == EWORKSPACE
    assert lib.grace_set_option(ctx, 99, 1) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_GRAPH_STEPS, 3) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_GRAPH_STEPS, 8) == 0
    assert lib.grace_set_film_hext(ctx, 1, _lib.dvec([0, 0, 0])) == EINVAL
    assert lib.grace_set_hext(ctx, _lib.dvec([1.0, 2.0, 3.0])) == 0
    assert lib.grace_destroy(ctx) == 0
    assert lib.grace_destroy(None) == 0


def test_batch_create_shares_tensor_per_shape(lib):
    grids = [(64, 16, 1), (128, 32, 1), (64, 16, 1), (200, 50, 1)]
    n = len(grids)
    ctx = C.c_void_p()
    st = lib.grace_batch_create(C.byref(ctx), n, _lib.ivec([g for t in grids for g in t]),
                                _lib.dvec([3e-9] * 3 * n), _lib.dvec([8e5] * n),
                                _lib.dvec([1.3e-11] * n), _lib.dvec([0.0] * n),
                                _lib.dvec([0.1] * n), _lib.dvec([2.211e5] * n))
    assert st == 0
    cnt = C.c_longlong()
    lib.grace_ncells(ctx, C.byref(cnt))
    assert cnt.value == sum(a * b * c for a, b, c in grids)
    lib.grace_destroy(ctx)
    bad = C.c_void_p()
    assert lib.grace_batch_create(C.byref(bad), 0, None, None, None, None, None, None, None) == EINVAL


def test_pulse_and_time_validation(lib):
    """Envelope times must be finite and non-decreasing; the time is kept on the host before
    grace_bind (no device call)."""
    st, ctx = _create(lib)
    assert st == 0
    for bad in ([1e-9, 0.5e-9, 2e-9], [0.0, 1e-9, 0.5e-9], [0.0, float("nan"), 1e-9],
                [0.0, 1e-9, float("inf")]):
        assert lib.grace_set_hext_pulse(ctx, _lib.dvec(bad)) == EINVAL
    assert lib.grace_set_hext_pulse(ctx, _lib.dvec([0.0, 1e-9, 1e-9])) == 0
    assert lib.grace_set_hext_pulse(ctx, None) == 0
    t = C.c_double()
    assert lib.grace_get_time(ctx, C.byref(t)) == 0 and t.value == 0.0
    assert lib.grace_set_time(ctx, 2.5e-10) == 0
    assert lib.grace_get_time(ctx, C.byref(t)) == 0 and t.value == 2.5e-10
    assert lib.grace_set_time(ctx, float("inf")) == EINVAL
    assert lib.grace_get_time(ctx, None) == EINVAL
    assert lib.grace_destroy(ctx) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without libgrace.so the binding raises instead of computing."""
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "libgrace.so"))


def test_batch_path_options_are_validated_on_the_host(lib):
    """GRACE_OPT_PERSISTENT is a planning option (before grace_bind, 0 or 1); the barrier
    bound and the failure-detection hook take their documented ranges; grace_sync needs a
    bound handle."""
    st, ctx = _create(lib)
    assert st == 0
    assert lib.grace_set_option(ctx, _lib.OPT_PERSISTENT, 1) == 0
    assert lib.grace_set_option(ctx, _lib.OPT_PERSISTENT, 2) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_PERSISTENT, 0) == 0
    assert lib.grace_set_option(ctx, _lib.OPT_BARRIER_TIMEOUT_US, 999) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_BARRIER_TIMEOUT_US, 200000) == 0
    assert lib.grace_set_option(ctx, _lib.OPT_TEST_SKIP_ARRIVE, -2) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_TEST_SKIP_ARRIVE, 3) == 0
    assert lib.grace_set_option(ctx, _lib.OPT_TEST_SKIP_ARRIVE, -1) == 0
    assert lib.grace_set_option(ctx, _lib.OPT_TILE_Z, 5) == EINVAL
    assert lib.grace_set_option(ctx, _lib.OPT_SIDE_STREAMS, 0) == 0
    assert lib.grace_sync(ctx) == ESTATE
    assert lib.grace_destroy(ctx) == 0
