"""Python face of the serving loop (include/svt.h, "Serving loop"): a
trigger-style server with continuous batching whose dispatcher, batching,
copies and latency accounting all run in libsvt.so (native thread, CUDA
streams and graphs).  This module only allocates the buffers (device memory
through PyTorch, pinned host memory) and marshals calls.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .api import _p


class Server:
    """Continuous-batching server over the fused path (mode 0) or the plain
    per-stage path (mode 1).  small_batch_events / small_blocks_per_sm: batches
    of at most that many events replay a second graph whose fit launch keeps
    fewer persistent blocks per SM (mode 0)."""

    def __init__(self, consts, n_slots=4, max_words=1 << 22, max_events=256, max_roads=1 << 16,
                 mode=0, max_combs=0, device_budget=0, max_queued_words=0, sched=None,
                 small_batch_events=0, small_blocks_per_sm=0, device="cuda"):
        L = N.load()
        self.consts = consts
        self.cfgs = N.SvtServerConfig(n_slots, mode, max_words, max_events, max_roads, max_combs,
                                      device_budget, max_queued_words, small_batch_events,
                                      small_blocks_per_sm)
        self.sched = sched
        d, h = ctypes.c_size_t(), ctypes.c_size_t()
        sp = ctypes.byref(sched) if sched is not None else None
        N.check(L.svt_server_sizes(ctypes.byref(self.cfgs), sp, ctypes.byref(d), ctypes.byref(h)),
                "svt_server_sizes")
        self.workspace = torch.empty(d.value, dtype=torch.uint8, device=device)
        self.pinned = torch.empty(h.value + 256, dtype=torch.uint8, pin_memory=True)
        base = self.pinned.data_ptr()
        self._pinned_ptr = ctypes.c_void_p((base + 255) // 256 * 256)
        h_handle = ctypes.c_void_p()
        torch.cuda.synchronize()
        N.check(L.svt_server_create(ctypes.byref(self.cfgs), _p(consts.F), _p(consts.q),
                                    ctypes.byref(consts.cfg), sp, _p(self.workspace),
                                    self.workspace.numel(), self._pinned_ptr, h.value,
                                    ctypes.byref(h_handle)), "svt_server_create")
        self.handle = h_handle
        self._keep = []

    def submit(self, h_words: torch.Tensor, tag: int, h_records: np.ndarray | None = None) -> int:
        """Queue one event whose words are a pinned host tensor (kept alive
        until its result arrives).  Returns the C status code."""
        rec = None if h_records is None else h_records.ctypes.data_as(ctypes.c_void_p)
        return N.load().svt_server_submit(self.handle, ctypes.c_void_p(h_words.data_ptr()),
                                          h_words.numel(), tag, rec)

    def poll(self, max_results=4096, wait_us=1000):
        buf = (N.SvtEventResult * max_results)()
        n = ctypes.c_uint32()
        N.check(N.load().svt_server_poll(self.handle, buf, max_results, ctypes.byref(n), wait_us),
                "svt_server_poll")
        return [buf[i] for i in range(n.value)]

    def stats(self):
        st = N.SvtServerStats()
        N.check(N.load().svt_server_stats_get(self.handle, ctypes.byref(st)), "svt_server_stats_get")
        return {f: getattr(st, f) for f, _ in N.SvtServerStats._fields_}

    def bench_poisson(self, h_pool: torch.Tensor, pool_off: np.ndarray, rate_hz: float,
                      n_events: int, seed: int = 1):
        """Poisson arrivals from a pinned pool of events; returns (latencies in
        ns as uint64, wall seconds)."""
        off = np.ascontiguousarray(pool_off, np.uint64)
        lat = np.zeros(n_events, np.uint64)
        wall = ctypes.c_double()
        rc = N.load().svt_server_bench_poisson(
            self.handle, ctypes.c_void_p(h_pool.data_ptr()), off.ctypes.data_as(ctypes.c_void_p),
            len(off) - 1, float(rate_hz), n_events, seed, lat.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(wall))
        N.check(rc, "svt_server_bench_poisson")
        return lat, wall.value

    def close(self):
        if getattr(self, "handle", None):
            N.load().svt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def pinned_pool(words: np.ndarray) -> torch.Tensor:
    """Pinned host copy of a word stream (uint32 -> int32 bits)."""
    return torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).pin_memory()
