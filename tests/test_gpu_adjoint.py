"""Adjoint LLG on the GPU (grace_backward) against the FP64 oracle's exact discrete adjoint.

The oracle adjoint is itself pinned by central finite differences of the FP64 forward map
(tests/test_oracle_pins.py).  The GPU runs FP32, so forward states differ from the
oracle's by rounding; gradients are compared in relative L2 norm (bar 1e-3)."""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint as oadj
from oracle import llg
from paper_1411_2565_gb300 import build as libbuild

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()


def _golden_module():
    """tests/golden/make_adjoint_film_4096.py, loaded by path (tests/ is not a package)."""
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_adjoint_film_4096.py")
    spec = importlib.util.spec_from_file_location("make_adjoint_film_4096", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def setup(grid, cell, steps, seed=5, Ku=0.0):
    from paper_1411_2565_gb300.grace import Grace
    f, m0 = workloads.small_film(grid, cell=cell, seed=seed, Ms=8e5, A=1.3e-11, Ku=Ku, alpha=0.1)
    shape = f.shape_zyx
    n = int(np.prod(shape))
    ms = (8e5 * (1 + 0.1 * (2 * workloads.uniform(seed + 1, n) - 1))).astype(np.float32).reshape(shape)
    h = (2e4 * (2 * workloads.uniform(seed + 2, 3 * n) - 1)).astype(np.float32).reshape((3,) + shape)
    target = workloads.smooth_target(shape, seed + 3)
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV)
    return f, m0, ms, h, target, g


def oracle_grads(f, m0, ms, h, target, dt, steps):
    p = llg.Params(f.cell, ms.astype(np.float64), f.A, f.Ku, f.alpha, f.gamma0, h.astype(np.float64))
    return oadj.gradients(m0, p, dt, steps, target)


@pytest.mark.parametrize("grid,steps,ckpt", [((24, 16, 2), 37, 8), ((20, 12, 1), 30, 30),
                                             ((12, 10, 6), 20, 7), ((4, 6, 3), 15, 4), ((3, 5, 2), 9, 1)])
def test_backward_matches_fp64_adjoint(grid, steps, ckpt):
    dt = 1e-14
    f, m0, ms, h, target, g = setup(grid, (4e-9, 4e-9, 3e-9), steps, Ku=2e3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    g.set_ms_field(dev(ms))
    g.set_hext_field(dev(h))
    g.set_m(dev(m0))
    g.step(steps, dt)
    mT = g.get_m()
    n = mT.numel() // 3
    lamT = 2.0 * (mT - dev(target)) / n
    g.set_m(dev(m0))
    gh = torch.zeros(3 * n, device=DEV)
    gms = torch.zeros(n, device=DEV)
    gm0 = g.backward(lamT, steps, dt, ckpt, gh, gms)
    loss, o_m0, o_h, o_ms = oracle_grads(f, m0, ms, h, target, dt, steps)
    assert rel(gh.cpu().numpy(), o_h) <= 1e-3
    assert rel(gms.cpu().numpy(), o_ms) <= 1e-3
    assert rel(gm0.cpu().numpy(), o_m0) <= 1e-3
    # the state is left at m_0
    assert torch.equal(g.get_m(), dev(m0))


def test_autograd_function_matches_direct_backward():
    from paper_1411_2565_gb300.autograd import llg as llg_fn
    dt, steps = 1e-14, 24
    f, m0, ms, h, target, g = setup((16, 12, 2), (4e-9, 4e-9, 3e-9), steps)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    m0t = dev(m0).requires_grad_(True)
    ht = dev(h).requires_grad_(True)
    mst = dev(ms).requires_grad_(True)
    mT = llg_fn(m0t, ht, mst, g, steps, dt, 10)
    loss = ((mT - dev(target)) ** 2).sum() / (mT.numel() // 3)
    loss.backward()
    _, o_m0, o_h, o_ms = oracle_grads(f, m0, ms, h, target, dt, steps)
    assert rel(ht.grad.cpu().numpy(), o_h) <= 1e-3
    assert rel(mst.grad.cpu().numpy(), o_ms) <= 1e-3
    assert rel(m0t.grad.cpu().numpy(), o_m0) <= 1e-3


def test_adjoint_workload_full_grid():
    """The 256x64x2 adjoint film (4x4x3 nm cells, per-cell Ms and field) for 128 steps with
    checkpoints every 64, against the FP64 adjoint."""
    w = workloads.adjoint_film()
    f, m0 = w.films[0], w.m0[0]
    from paper_1411_2565_gb300.grace import Grace
    steps, dt = 128, w.dt
    shape = f.shape_zyx
    ms = w.ms_field
    h = np.zeros((3,) + shape, dtype=np.float32)
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    g.set_ms_field(dev(ms))
    g.set_hext_field(dev(h))
    g.set_m(dev(m0))
    g.step(steps, dt)
    mT = g.get_m()
    n = mT.numel() // 3
    lamT = 2.0 * (mT - dev(w.target)) / n
    g.set_m(dev(m0))
    gh = torch.zeros(3 * n, device=DEV)
    gms = torch.zeros(n, device=DEV)
    gm0 = g.backward(lamT, steps, dt, 64, gh, gms)
    _, o_m0, o_h, o_ms = oracle_grads(f, m0, ms, h, w.target, dt, steps)
    assert rel(gh.cpu().numpy(), o_h) <= 1e-3
    assert rel(gms.cpu().numpy(), o_ms) <= 1e-3
    assert rel(gm0.cpu().numpy(), o_m0) <= 1e-3


def test_adjoint_workload_stated_length():
    """The adjoint workload at its stated length: 4,096 Euler steps on the 256x64x2 film
    with checkpoints every 64 (64 recomputed segments), gradients w.r.t. the per-cell
    applied field, the per-cell Ms and m_0 against the FP64 oracle adjoint of the same
    4,096 steps (tests/golden/adjoint_film_4096.npz, written by make_adjoint_film_4096.py
    from the oracle alone)."""
    gm = _golden_module()
    OUT, STEPS, inputs_digest = gm.OUT, gm.STEPS, gm.inputs_digest
    from paper_1411_2565_gb300.grace import Grace
    w = workloads.adjoint_film()
    gold = np.load(OUT)
    assert str(gold["digest"]) == inputs_digest(w), "fixture out of date: rerun its script"
    f, m0 = w.films[0], w.m0[0]
    dt, shape = w.dt, f.shape_zyx
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    g.set_ms_field(dev(w.ms_field))
    g.set_hext_field(dev(np.zeros((3,) + shape, dtype=np.float32)))
    g.set_m(dev(m0))
    g.step(STEPS, dt)
    mT = g.get_m()
    n = mT.numel() // 3
    loss = float(((mT.double() - dev(w.target).double()) ** 2).sum() / n)
    assert abs(loss - float(gold["loss"])) <= 1e-4 * abs(float(gold["loss"]))
    lamT = 2.0 * (mT - dev(w.target)) / n
    g.set_m(dev(m0))
    gh = torch.zeros(3 * n, device=DEV)
    gms = torch.zeros(n, device=DEV)
    gm0 = g.backward(lamT, STEPS, dt, 64, gh, gms)
    assert rel(gh.cpu().numpy(), gold["g_hext"]) <= 1e-3
    assert rel(gms.cpu().numpy(), gold["g_ms"]) <= 1e-3
    assert rel(gm0.cpu().numpy(), gold["g_m0"]) <= 1e-3


def test_backward_graph_replay_equals_direct_launches():
    """grace_backward replays captured graphs of its forward runs and of each segment's
    recompute + backward; with graphs off the same launches run directly.  Both give the
    same gradients bit for bit, also when the checkpoint interval leaves a short, odd last
    segment (41 = 3 x 12 + 5 steps)."""
    dt, steps, ckpt = 1e-14, 41, 12
    f, m0, ms, h, target, g = setup((24, 16, 2), (4e-9, 4e-9, 3e-9), steps, Ku=2e3)
    from paper_1411_2565_gb300 import _lib
    from paper_1411_2565_gb300.grace import Grace
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    outs = []
    for graph in (1, 0):
        gg = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV,
                   options={_lib.OPT_GRAPH: graph})
        gg.set_ms_field(dev(ms))
        gg.set_hext_field(dev(h))
        gg.set_m(dev(m0))
        n = 3 * f.ncells
        lam = torch.linspace(-1e-3, 1e-3, n, device=DEV)
        gh = torch.zeros(n, device=DEV)
        gms = torch.zeros(f.ncells, device=DEV)
        gm0 = gg.backward(lam, steps, dt, ckpt, gh, gms)
        outs.append((gh, gms, gm0, gg.get_m()))
        gg.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert torch.equal(outs[0][3], dev(m0))          # the state is left at m_0


def test_checkpointed_forward_and_backward_equal_the_plain_calls():
    """grace_step_checkpointed ends at the state grace_step reaches, and the adjoint from its
    checkpoints (grace_backward_checkpointed) equals grace_backward, which collects the
    same checkpoints in a forward pass of its own, bit for bit (41 = 3 x 12 + 5 steps)."""
    dt, steps, ckpt = 1e-14, 41, 12
    f, m0, ms, h, target, g = setup((24, 16, 2), (4e-9, 4e-9, 3e-9), steps, Ku=2e3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    g.set_ms_field(dev(ms))
    g.set_hext_field(dev(h))
    g.set_m(dev(m0))
    tape = g.step_checkpointed(steps, dt, ckpt)
    m_tape = g.get_m()
    g.set_m(dev(m0))
    g.step(steps, dt)
    assert torch.equal(m_tape, g.get_m())
    n = 3 * f.ncells
    lam = torch.linspace(-1e-3, 1e-3, n, device=DEV)
    outs = []
    for use_tape in (False, True):
        g.set_m(dev(m0) if not use_tape else m_tape)
        gh = torch.zeros(n, device=DEV)
        gms = torch.zeros(f.ncells, device=DEV)
        gm0 = g.backward(lam, steps, dt, ckpt, gh, gms, tape=tape if use_tape else None)
        outs.append((gh, gms, gm0, g.get_m()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    assert torch.equal(outs[1][3], dev(m0))          # the state is left at m_0
    with pytest.raises(ValueError):
        g.backward(lam, steps, dt, ckpt + 1, tape=tape)
    g.close()


@pytest.mark.parametrize("tile_x", [1, 2])
def test_backward_on_the_x_tiles_of_px_512(tile_x):
    """The adjoint x-pass modes on one line per block (with helper warps) and on the 4-line
    tile (Px = 512), against the FP64 adjoint."""
    from paper_1411_2565_gb300 import _lib
    from paper_1411_2565_gb300.grace import Grace
    dt, steps, ckpt = 1e-14, 11, 4
    f, m0, ms, h, target, g0 = setup((140, 9, 2), (4e-9, 4e-9, 3e-9), steps, Ku=2e3)
    g0.close()
    g = Grace(f.grid, f.cell, f.Ms, f.A, f.Ku, f.alpha, f.gamma0, device=DEV, options={_lib.OPT_TILE_X: tile_x})
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(DEV)
    g.set_ms_field(dev(ms))
    g.set_hext_field(dev(h))
    g.set_m(dev(m0))
    tape = g.step_checkpointed(steps, dt, ckpt)
    mT = g.get_m()
    n = mT.numel() // 3
    lamT = 2.0 * (mT - dev(target)) / n
    gh = torch.zeros(3 * n, device=DEV)
    gms = torch.zeros(n, device=DEV)
    gm0 = g.backward(lamT, steps, dt, ckpt, gh, gms, tape=tape)
    loss, o_m0, o_h, o_ms = oracle_grads(f, m0, ms, h, target, dt, steps)
    assert rel(gh.cpu().numpy(), o_h) <= 1e-3
    assert rel(gms.cpu().numpy(), o_ms) <= 1e-3
    assert rel(gm0.cpu().numpy(), o_m0) <= 1e-3
    g.close()
