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

    def reset_stats(self):
        N.check(N.load().svt_server_stats_reset(self.handle), "svt_server_stats_reset")

    def trace_start(self, cap: int = 1 << 20, device_times: bool = True):
        """Record one entry per completed batch (up to cap) until trace_stop;
        device_times adds each batch's device interval (two timing events)."""
        self._trace = (N.SvtBatchTrace * cap)()
        N.check(N.load().svt_server_trace(self.handle, ctypes.cast(self._trace, ctypes.c_void_p),
                                          cap, int(device_times)), "svt_server_trace")

    def trace_stop(self) -> np.ndarray:
        """Stops the trace; returns its entries as a structured array."""
        L = N.load()
        n = ctypes.c_uint64()
        N.check(L.svt_server_trace(self.handle, None, 0, 0), "svt_server_trace")
        N.check(L.svt_server_trace_count(self.handle, ctypes.byref(n)), "svt_server_trace_count")
        buf = getattr(self, "_trace", None)
        self._trace = None
        if buf is None:
            return np.zeros(0, dtype=TRACE_DTYPE)
        raw = np.frombuffer(buf, dtype=TRACE_DTYPE)
        return raw[:min(int(n.value), len(raw))].copy()

    def bench_poisson(self, h_pool: torch.Tensor, pool_off: np.ndarray, rate_hz: float,
                      n_events: int, seed: int = 1, records: np.ndarray | None = None,
                      rec_off: np.ndarray | None = None):
        """Poisson arrivals from a pinned pool of events (event i is pool event
        i mod pool size); returns (latencies in ns from each scheduled arrival
        as uint64, wall seconds).  records / rec_off: event i's records land at
        records[rec_off[i]:] (rows of 6 words)."""
        off = np.ascontiguousarray(pool_off, np.uint64)
        lat = np.zeros(n_events, np.uint64)
        wall = ctypes.c_double()
        rp = ro = None
        if records is not None:
            assert records.dtype == np.uint32 and records.flags.c_contiguous
            ro_arr = np.ascontiguousarray(rec_off, np.uint64)
            assert len(ro_arr) >= n_events
            rp = records.ctypes.data_as(ctypes.c_void_p)
            ro = ro_arr.ctypes.data_as(ctypes.c_void_p)
        rc = N.load().svt_server_bench_poisson(
            self.handle, ctypes.c_void_p(h_pool.data_ptr()), off.ctypes.data_as(ctypes.c_void_p),
            len(off) - 1, float(rate_hz), n_events, seed, rp, ro,
            lat.ctypes.data_as(ctypes.c_void_p), ctypes.byref(wall))
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


TRACE_DTYPE = np.dtype([("slot", np.uint32), ("n_events", np.uint32), ("n_roads", np.uint32),
                        ("queued_after", np.uint32), ("t_first_arrive_ns", np.int64),
                        ("t_dispatch_ns", np.int64), ("t_enqueued_ns", np.int64),
                        ("t_done_ns", np.int64), ("dev_start_us", np.float32),
                        ("dev_end_us", np.float32)])


def overlap_fraction(trace: np.ndarray) -> float:
    """Fraction of traced batches whose device interval (first copy in to last
    copy out) overlaps the interval of a batch in another slot."""
    t = trace[(trace["dev_start_us"] >= 0) & (trace["dev_end_us"] >= 0)]
    if len(t) < 2:
        return 0.0
    order = np.argsort(t["dev_start_us"], kind="stable")
    a, z, s = t["dev_start_us"][order], t["dev_end_us"][order], t["slot"][order]
    hit = np.zeros(len(t), bool)
    for i in range(len(t)):
        j = i + 1
        while j < len(t) and a[j] < z[i]:
            if s[j] != s[i]:
                hit[i] = hit[j] = True
            j += 1
    return float(hit.mean())


def pinned_pool(words: np.ndarray) -> torch.Tensor:
    """Pinned host copy of a word stream (uint32 -> int32 bits)."""
    return torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).pin_memory()
