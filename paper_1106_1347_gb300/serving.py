"""Python driver for libmm's serving loop (mm_server_* in include/mm.h).

The server itself -- admission under the HBM budget, continuous batching,
grouped launches replayed from CUDA graphs, completion tracking -- runs in the
library's native worker thread; this module only marshals requests and reads
completions and statistics.  `replay` drives a trace with Poisson arrivals.
"""
from __future__ import annotations

import ctypes
import gc
import time

from ._native import Completion, Request, ServerStats, check, lib

i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p


Stats = ServerStats


def _declare():
    return lib()


METHOD_EMULATED = 0       # BF16 slices
METHOD_FP64 = 1           # one request at a time with the plain FP64 kernel (baseline)
METHOD_EMULATED_AUTO = 2  # per request the cheaper of BF16 and FP8-E4M3 slices for its tier


class Server:
    """A serving loop on one device with an HBM budget of `arena_bytes`."""

    def __init__(self, arena_bytes: int, max_batch: int = 64, nstreams: int = 4, use_graphs: bool = True,
                 method: int = METHOD_EMULATED, device=None):
        import torch

        self._L = _declare()
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        self._keep = {}  # host buffers of in-flight requests, by tag
        h = vp()
        check("mm_server_create", self._L.mm_server_create(ctypes.c_void_p(self.arena.data_ptr()), int(arena_bytes),
                                                           max_batch, nstreams, int(use_graphs), method,
                                                           ctypes.byref(h)))
        self._h = h

    @staticmethod
    def _hptr(x):
        import numpy as np
        import torch

        if isinstance(x, torch.Tensor):
            if x.is_cuda or x.dtype != torch.float64 or x.dim() != 2 or x.stride(1) != 1:
                raise TypeError("host operands must be 2-D float64 CPU tensors with unit column stride")
            return x.data_ptr(), max(1, x.stride(0) if x.shape[0] > 1 else x.shape[1]), tuple(x.shape)
        x = np.asarray(x)
        if x.dtype != np.float64 or x.ndim != 2 or x.strides[1] != 8:
            raise TypeError("host operands must be 2-D float64 arrays with unit column stride")
        return x.ctypes.data, max(1, x.strides[0] // 8 if x.shape[0] > 1 else x.shape[1]), x.shape

    def submit(self, a, b, c, tier: float = 1e-14, tag: int = 0) -> None:
        """Queue C = A B (host buffers; keep them alive until the completion)."""
        pa, lda, sa = self._hptr(a)
        pb, ldb, sb = self._hptr(b)
        pc, ldc, sc = self._hptr(c)
        if sa[1] != sb[0] or sc != (sa[0], sb[1]):
            raise ValueError("shape mismatch")
        r = Request(sa[0], sa[1], sb[1], pa, lda, pb, ldb, pc, ldc, float(tier), int(tag))
        self._keep[int(tag)] = (a, b, c)
        rc = self._L.mm_server_submit(self._h, ctypes.byref(r))
        if rc != 0:
            self._keep.pop(int(tag), None)
            check("mm_server_submit", rc)

    def poll(self, cap: int = 4096):
        buf = (Completion * cap)()
        n = self._L.mm_server_poll(self._h, buf, cap)
        if n < 0:
            check("mm_server_poll", n)
        out = []
        for i in range(n):
            c = buf[i]
            self._keep.pop(int(c.tag), None)
            out.append({"tag": int(c.tag), "status": int(c.status), "slices": int(c.slices), "kind": int(c.kind),
                        "queue_ms": float(c.queue_ms), "latency_ms": float(c.latency_ms)})
        return out

    def wait(self, timeout_s: float = 600.0) -> int:
        return int(self._L.mm_server_wait(self._h, int(timeout_s * 1000)))

    def error(self) -> str:
        msg = self._L.mm_server_error(self._h)
        return msg.decode() if msg else ""

    def stats(self) -> dict:
        st = Stats()
        check("mm_server_stats", self._L.mm_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def close(self) -> int:
        if self._h is not None:
            rc = int(self._L.mm_server_destroy(self._h))
            self._h = None
            self._keep.clear()
            return rc
        return 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def replay(server: Server, trace, a_pool, b_pool, c_pool, time_scale: float = 1.0, check_every: int = 0):
    """Submit `trace` (dicts with arrival_s, N, P, M, tier, id) at its arrival
    times; operands are views of the pinned pools (A = a_pool[:N, :P], ...).
    Each request writes its own region of c_pool (rows of width M, starting at
    row (id * 1117) mod capacity), so concurrent requests rarely alias.
    Returns (stats, completions)."""
    rows_c = c_pool.shape[0] * c_pool.shape[1]
    flat_c = c_pool.view(-1)
    # A full collection of a large Python heap stalls the submitting thread for
    # tens of milliseconds, which would arrive as a burst of late requests: the
    # collector stays off while the trace is submitted.
    gc.collect()
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for req in trace:
            due = t0 + req["arrival_s"] * time_scale
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 2e-3:
                    time.sleep(due - now - 1e-3)
            n, p, m = req["N"], req["P"], req["M"]
            start = (req["id"] * 1117 * 4096) % max(1, rows_c - n * m)
            c = flat_c[start: start + n * m].view(n, m)
            server.submit(a_pool[:n, :p], b_pool[:p, :m], c, tier=req["tier"], tag=req["id"])
    finally:
        if was_enabled:
            gc.enable()
    rc = server.wait()
    comps = server.poll(len(trace) + 16)
    if rc != 0:
        raise RuntimeError(f"serving failed with status {rc}: {server.error()}")
    return server.stats(), comps, rc
