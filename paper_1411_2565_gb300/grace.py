"""Python binding of the C ABI: ``Grace`` (one film) and ``GraceBatch`` (an ensemble).

PyTorch supplies device memory (the workspace and I/O tensors) and the CUDA stream;
every step of the computation runs in libgrace.so.  Field tensors are FP32
``[3, nz, ny, nx]`` per film (a batch uses one flat tensor: films concatenated).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import TERM_ALL, check, dvec, ivec

GAMMA0 = 2.211e5


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t: torch.Tensor, numel: int, what: str) -> int:
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous float32 CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{what}: expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


class _Base:
    def _init(self, ctx: C.c_void_p, device, stream, options=None):
        self._L = _lib.load()
        self.ctx = ctx
        for opt, val in (options or {}).items():      # tile options must precede the bind
            check(self._L.grace_set_option(ctx, int(opt), int(val)), "grace_set_option", ctx)
        self.device = torch.device(device)
        n = C.c_longlong()
        check(self._L.grace_ncells(ctx, C.byref(n)), "grace_ncells", ctx)
        self.ncell = int(n.value)
        sz = C.c_size_t()
        check(self._L.grace_workspace_size(ctx, C.byref(sz)), "grace_workspace_size", ctx)
        self.workspace_bytes = int(sz.value)
        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                     device=self.device)
        self.stream = stream
        if stream is not None:
            # the handle's work runs on `stream`: the allocator must not hand the workspace
            # out again before that work is done
            self.workspace.record_stream(stream)
        check(self._L.grace_bind(ctx, self.workspace.data_ptr(), self.workspace_bytes,
                                 _stream_ptr(stream)), "grace_bind", ctx)
        self._keep = {}

    # -- state ------------------------------------------------------------------
    def set_m(self, m: torch.Tensor):
        check(self._L.grace_set_m(self.ctx, _dev_ptr(m, 3 * self.ncell, "m")), "grace_set_m", self.ctx)

    def get_m(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(3 * self.ncell, dtype=torch.float32, device=self.device)
            if self.stream is not None:
                out.record_stream(self.stream)   # written on the handle's stream
        check(self._L.grace_get_m(self.ctx, _dev_ptr(out, 3 * self.ncell, "out")), "grace_get_m",
              self.ctx)
        return out

    def set_m_host(self, m: np.ndarray):
        a = np.ascontiguousarray(m, dtype=np.float32)
        if a.size != 3 * self.ncell:
            raise ValueError("m: wrong size")
        check(self._L.grace_set_m_host(self.ctx, a.ctypes.data), "grace_set_m_host", self.ctx)
        self._keep["m_host"] = a   # the copy is queued; keep the buffer alive

    def get_m_host(self, out: Optional[np.ndarray] = None, wait: bool = True) -> np.ndarray:
        """Copy m to host memory; with wait=False the copy is only queued on the handle's
        stream (grace_get_m_host_async): `out` (page-locked) is valid after a stream sync."""
        if out is None:
            out = np.empty(3 * self.ncell, dtype=np.float32)
        if wait:
            check(self._L.grace_get_m_host(self.ctx, out.ctypes.data), "grace_get_m_host", self.ctx)
        else:
            check(self._L.grace_get_m_host_async(self.ctx, out.ctypes.data), "grace_get_m_host_async", self.ctx)
        return out

    # -- parameters ---------------------------------------------------------------
    def set_hext(self, h: Sequence[float]):
        check(self._L.grace_set_hext(self.ctx, dvec(h)), "grace_set_hext", self.ctx)

    def set_hext_field(self, h: Optional[torch.Tensor]):
        ptr = None if h is None else _dev_ptr(h, 3 * self.ncell, "hext field")
        check(self._L.grace_set_hext_field(self.ctx, ptr), "grace_set_hext_field", self.ctx)
        self._keep["h"] = h

    def set_ms_field(self, ms: Optional[torch.Tensor]):
        ptr = None if ms is None else _dev_ptr(ms, self.ncell, "Ms field")
        check(self._L.grace_set_ms_field(self.ctx, ptr), "grace_set_ms_field", self.ctx)
        self._keep["ms"] = ms

    def set_hext_pulse(self, times: Optional[Sequence[float]]):
        """Applied-field envelope (t_start, t_decay, t_stop) in s, or None for a constant field
        (grace_set_hext_pulse)."""
        arg = None if times is None else dvec(times)
        check(self._L.grace_set_hext_pulse(self.ctx, arg), "grace_set_hext_pulse", self.ctx)

    @property
    def time(self) -> float:
        t = C.c_double()
        check(self._L.grace_get_time(self.ctx, C.byref(t)), "grace_get_time", self.ctx)
        return t.value

    @time.setter
    def time(self, t: float):
        check(self._L.grace_set_time(self.ctx, float(t)), "grace_set_time", self.ctx)

    def trace(self, capacity: int = 1 << 16):
        """Time the next ``capacity`` kernel launches with CUDA events (0 switches it off)."""
        check(self._L.grace_trace(self.ctx, int(capacity)), "grace_trace", self.ctx)

    def trace_read(self):
        """{kernel kind: (total ms, launches)} since the last read (see GRACE_KERNEL_*)."""
        ms = (C.c_double * 8)()
        n = (C.c_longlong * 8)()
        check(self._L.grace_trace_read(self.ctx, ms, n), "grace_trace_read", self.ctx)
        return {name: (ms[k], int(n[k])) for k, name in enumerate(_lib.KERNEL_NAMES) if n[k]}

    def set_option(self, option: int, value: int):
        check(self._L.grace_set_option(self.ctx, option, value), "grace_set_option", self.ctx)

    def sync(self):
        """Wait for the handle's stream; raises GraceError (GRACE_ETIMEOUT) if a grid barrier of
        the persistent batch launch timed out since the last report (grace_sync)."""
        check(self._L.grace_sync(self.ctx), "grace_sync", self.ctx)

    # -- compute ------------------------------------------------------------------
    def heff(self, mask: int = TERM_ALL, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(3 * self.ncell, dtype=torch.float32, device=self.device)
            if self.stream is not None:
                out.record_stream(self.stream)   # written on the handle's stream
        check(self._L.grace_heff(self.ctx, _dev_ptr(out, 3 * self.ncell, "out"), mask), "grace_heff",
              self.ctx)
        return out

    def step(self, n: int, dt: float):
        check(self._L.grace_step(self.ctx, int(n), float(dt)), "grace_step", self.ctx)

    def _scratch(self, n: int, ckpt_every: int):
        sz = C.c_size_t()
        check(self._L.grace_backward_workspace_size(self.ctx, int(n), int(ckpt_every), C.byref(sz)),
              "grace_backward_workspace_size", self.ctx)
        scratch = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=self.device)
        if self.stream is not None:
            scratch.record_stream(self.stream)
        return scratch, int(sz.value)

    def step_checkpointed(self, n: int, dt: float, ckpt_every: int = 64) -> "Tape":
        """``n`` Euler steps as ``step`` that also keep every ``ckpt_every``-th state
        (grace_step_checkpointed); ``backward(..., tape=)`` then skips its own forward pass."""
        scratch, nbytes = self._scratch(n, ckpt_every)
        check(self._L.grace_step_checkpointed(self.ctx, int(n), float(dt), int(ckpt_every),
                                              scratch.data_ptr(), nbytes), "grace_step_checkpointed", self.ctx)
        return Tape(scratch, nbytes, int(n), float(dt), int(ckpt_every))

    def backward(self, dL_dmT: torch.Tensor, n: int, dt: float, ckpt_every: int = 64,
                 g_hext: Optional[torch.Tensor] = None, g_ms: Optional[torch.Tensor] = None,
                 want_m0: bool = True, tape: Optional["Tape"] = None) -> Optional[torch.Tensor]:
        """Discrete adjoint of ``n`` Euler steps (grace_backward): from the current state, or
        with ``tape`` from the checkpoints of ``step_checkpointed`` (same n, dt, ckpt_every;
        grace_backward_checkpointed).

        Adds dL/dH_ext into ``g_hext`` (3N) and dL/dMs into ``g_ms`` (N) when given and
        returns dL/dm_0; the state is left at m_0."""
        if tape is not None:
            if (tape.n, tape.dt, tape.ckpt_every) != (int(n), float(dt), int(ckpt_every)):
                raise ValueError("the tape was recorded with another n, dt or ckpt_every")
            scratch, nbytes = tape.scratch, tape.nbytes
            fn, name = self._L.grace_backward_checkpointed, "grace_backward_checkpointed"
        else:
            scratch, nbytes = self._scratch(n, ckpt_every)
            fn, name = self._L.grace_backward, "grace_backward"
        gm0 = torch.empty(3 * self.ncell, dtype=torch.float32, device=self.device) if want_m0 else None
        if self.stream is not None and gm0 is not None:
            gm0.record_stream(self.stream)
        check(fn(self.ctx, _dev_ptr(dL_dmT, 3 * self.ncell, "dL/dm_T"), int(n), float(dt), int(ckpt_every),
                 scratch.data_ptr(), nbytes,
                 None if g_hext is None else _dev_ptr(g_hext, 3 * self.ncell, "g_hext"),
                 None if g_ms is None else _dev_ptr(g_ms, self.ncell, "g_ms"),
                 None if gm0 is None else gm0.data_ptr()), name, self.ctx)
        return gm0

    def energy(self):
        e = (C.c_double * 5)()
        mv = (C.c_double * 3)()
        check(self._L.grace_energy(self.ctx, e, mv), "grace_energy", self.ctx)
        names = ("exch", "anis", "demag", "zeeman", "total")
        return dict(zip(names, list(e))), np.array(list(mv))

    def close(self):
        """Release the handle (its streams, events and graphs); the tensors stay with torch."""
        if getattr(self, "ctx", None):
            self._L.grace_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Shape:
    """A film's grid and cell, as the autotuner keys them."""

    def __init__(self, grid, cell):
        self.grid = tuple(int(g) for g in grid)
        self.cell = tuple(float(c) for c in cell)


def _tuned(films, device, options, tuned):
    """options as given; with options None and tuned, the autotuner's schedule for these
    films (its cache, else the shipped GB300 table, else {}: the library's heuristics)."""
    if options is not None or not tuned:
        return dict(options or {})
    from . import autotune
    return autotune.best(films, device)


class Tape:
    """Checkpoints written by ``Grace.step_checkpointed``: the device scratch and the
    (n, dt, ckpt_every) they were taken with."""

    def __init__(self, scratch: torch.Tensor, nbytes: int, n: int, dt: float, ckpt_every: int):
        self.scratch, self.nbytes, self.n, self.dt, self.ckpt_every = scratch, nbytes, n, dt, ckpt_every


class Grace(_Base):
    """One rectangular film (grid (nx, ny, nz), cell (dx, dy, dz) in metres).

    ``options`` (GRACE_OPT_* -> value) are applied before the bind; by default (None) the
    autotuned schedule for this shape is, unless ``tuned=False``.  ``self.options`` holds
    what was applied."""

    def __init__(self, grid, cell, Ms, A, Ku=0.0, alpha=0.1, gamma0=GAMMA0, device="cuda",
                 stream: Optional[torch.cuda.Stream] = None, options=None, tuned=True):
        L = _lib.load()
        ctx = C.c_void_p()
        check(L.grace_create(C.byref(ctx), ivec(grid), dvec(cell), float(Ms), float(A), float(Ku),
                             float(alpha), float(gamma0)), "grace_create")
        self.grid = tuple(int(g) for g in grid)
        self.options = _tuned([_Shape(grid, cell)], device, options, tuned)
        self._init(ctx, device, stream, self.options)

    @property
    def shape(self):
        nx, ny, nz = self.grid
        return (3, nz, ny, nx)


class GraceBatch(_Base):
    """Independent films stepped together; arrays are the films concatenated in order.
    ``options`` and ``tuned`` as for ``Grace``."""

    def __init__(self, films, device="cuda", stream: Optional[torch.cuda.Stream] = None, options=None,
                 tuned=True):
        L = _lib.load()
        ctx = C.c_void_p()
        n = len(films)
        grid = [g for f in films for g in f.grid]
        cell = [c for f in films for c in f.cell]
        check(L.grace_batch_create(C.byref(ctx), n, ivec(grid), dvec(cell),
                                   dvec([f.Ms for f in films]), dvec([f.A for f in films]),
                                   dvec([f.Ku for f in films]), dvec([f.alpha for f in films]),
                                   dvec([f.gamma0 for f in films])), "grace_batch_create")
        self.films = list(films)
        self.options = _tuned(self.films, device, options, tuned)
        self._init(ctx, device, stream, self.options)
        for i, f in enumerate(films):
            check(L.grace_set_film_hext(ctx, i, dvec(f.hext)), "grace_set_film_hext", ctx)
        self.offsets = np.cumsum([0] + [3 * f.ncells for f in films])

    def split(self, flat: torch.Tensor):
        """Per-film views [3, nz, ny, nx] of a concatenated field."""
        return [flat[self.offsets[i]:self.offsets[i + 1]].view(3, f.grid[2], f.grid[1], f.grid[0])
                for i, f in enumerate(self.films)]
