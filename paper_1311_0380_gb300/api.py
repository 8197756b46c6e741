"""Python face of the C ABI: the same names as include/svt.h, plus two small
holders that own device buffers (allocated through PyTorch) for the plain and
the fused path.  Nothing here computes any part of the fit: every step runs in
libsvt.so's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

SvtConfig = N.SvtConfig
SvtSchedule = N.SvtSchedule


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def config(oshift=15, qshift=15, chi2_cut=0xFFFFFFFF, max_comb=262144, min_layers=5,
           n_sectors=512, xft_pairs=0) -> SvtConfig:
    return SvtConfig(oshift, qshift, chi2_cut, max_comb, min_layers, n_sectors, xft_pairs)


def schedule(warps_per_block=0, blocks_per_sm=0, rows_per_item=0, roads_per_chunk=0,
             small_max=0, pair_small=0) -> SvtSchedule:
    return SvtSchedule(warps_per_block, blocks_per_sm, rows_per_item, roads_per_chunk, small_max,
                       pair_small)


# ------------------------------------------------------------------ raw entry points
def svt_version() -> int:
    return N.load().svt_version()


def pipe_peak(mode: int, iters: int = 1 << 14, stream=None):
    """Measured arithmetic throughput of the current GPU (svt_pipe_peak):
    returns (operations per second, seconds of the timed launch).  mode 0:
    int32 3-input adds, 1: int32 multiply-adds, 2: both, 3: fp32 multiply and
    fused multiply-add (the issue rate)."""
    ops, sec = ctypes.c_double(), ctypes.c_double()
    N.check(N.load().svt_pipe_peak(mode, iters, ctypes.byref(ops), ctypes.byref(sec),
                                   _stream(stream)), "svt_pipe_peak")
    return ops.value, sec.value


def svt_device_sm_count(device: int = 0) -> int:
    return N.load().svt_device_sm_count(device)


def svt_unpack_workspace_size(n_words: int) -> int:
    return N.load().svt_unpack_workspace_size(n_words)


def svt_unpack(words, n_words, event_off, n_events, n_sectors, road_cap, road_word, road_nhit,
               event_road, n_roads, status, workspace, stream=None, xft_pairs=0):
    N.check(N.load().svt_unpack(_p(words), n_words, _p(event_off), n_events, n_sectors, xft_pairs,
                                road_cap, _p(road_word), _p(road_nhit), _p(event_road),
                                _p(n_roads), _p(status), _p(workspace), workspace.numel(),
                                _stream(stream)),
            "svt_unpack")


def svt_combine_workspace_size(road_cap: int) -> int:
    return N.load().svt_combine_workspace_size(road_cap)


def svt_combine(road_nhit, n_roads, road_cap, cfg, comb_cap, road_flags, comb_off, comb_road,
                comb_hits, n_combs, status, workspace, stream=None):
    N.check(N.load().svt_combine(_p(road_nhit), _p(n_roads), road_cap, ctypes.byref(cfg), comb_cap,
                                 _p(road_flags), _p(comb_off), _p(comb_road), _p(comb_hits),
                                 _p(n_combs), _p(status), _p(workspace), workspace.numel(),
                                 _stream(stream)), "svt_combine")


def svt_fit(words, road_word, road_nhit, comb_road, comb_hits, n_combs, comb_cap, F, q, cfg,
            fit_chi2, fit_par, status, stream=None):
    N.check(N.load().svt_fit(_p(words), _p(road_word), _p(road_nhit), _p(comb_road),
                             _p(comb_hits), _p(n_combs), comb_cap, _p(F), _p(q), ctypes.byref(cfg),
                             _p(fit_chi2), _p(fit_par), _p(status), _stream(stream)), "svt_fit")


def svt_select(fit_chi2, fit_par, comb_cap, comb_off, road_flags, n_roads, road_cap, cfg, best,
               status, stream=None):
    N.check(N.load().svt_select(_p(fit_chi2), _p(fit_par), comb_cap, _p(comb_off), _p(road_flags),
                                _p(n_roads), road_cap, ctypes.byref(cfg), _p(best), _p(status),
                                _stream(stream)), "svt_select")


def svt_format(best, words, road_word, n_roads, road_cap, out, status, stream=None):
    N.check(N.load().svt_format(_p(best), _p(words), _p(road_word), _p(n_roads), road_cap,
                                _p(out), _p(status), _stream(stream)), "svt_format")


def svt_run_workspace_size(max_words, max_events, road_cap, sched=None) -> int:
    return N.load().svt_run_workspace_size(max_words, max_events, road_cap,
                                           ctypes.byref(sched) if sched is not None else None)


def svt_run(words, n_words, event_off, n_events, F, q, cfg, road_cap, out, event_road, counts,
            status, workspace, sched=None, timer=None, stream=None):
    N.check(N.load().svt_run(_p(words), n_words, _p(event_off), n_events, _p(F), _p(q),
                             ctypes.byref(cfg), road_cap, _p(out), _p(event_road), _p(counts),
                             _p(status), _p(workspace), workspace.numel(),
                             ctypes.byref(sched) if sched is not None else None,
                             timer.handle if timer is not None else None,
                             _stream(stream)), "svt_run")


def svt_run_noalloc(words, n_words, event_off, n_events, F, q, cfg, road_cap, out, event_road,
                    counts, status, sched=None, stream=None):
    """svt_run for callers that cannot allocate device memory: the scratch is
    a fixed array inside libsvt.so (svt_run_noalloc_scratch_bytes() per GPU),
    shared by every call on that GPU, so calls must not overlap on the device."""
    N.check(N.load().svt_run_noalloc(_p(words), n_words, _p(event_off), n_events, _p(F), _p(q),
                                     ctypes.byref(cfg), road_cap, _p(out), _p(event_road),
                                     _p(counts), _p(status),
                                     ctypes.byref(sched) if sched is not None else None,
                                     _stream(stream)), "svt_run_noalloc")


class FitTimer:
    """CUDA events recorded by svt_run around its persistent fit kernel."""

    def __init__(self):
        h = ctypes.c_void_p()
        N.check(N.load().svt_timer_create(ctypes.byref(h)), "svt_timer_create")
        self.handle = h

    def fit_ms(self) -> float:
        ms = ctypes.c_float()
        N.check(N.load().svt_timer_fit_ms(self.handle, ctypes.byref(ms)), "svt_timer_fit_ms")
        return float(ms.value)

    def __del__(self):
        try:
            if self.handle:
                N.load().svt_timer_destroy(self.handle)
                self.handle = None
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------------------ helpers
def to_device_u32(a: np.ndarray, device="cuda") -> torch.Tensor:
    """uint32 numpy -> int32 device tensor holding the same bits (16-byte aligned)."""
    a = np.ascontiguousarray(a, np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def to_device_u64(a: np.ndarray, device="cuda") -> torch.Tensor:
    a = np.ascontiguousarray(a, np.uint64)
    return torch.from_numpy(a.view(np.int64)).to(device)


def to_device_i16(a: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, np.int16)).to(device)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def roads_in(words: np.ndarray, event_off: np.ndarray) -> int:
    """Road count stated by the event headers (host side, O(events))."""
    if len(event_off) <= 1 or len(words) == 0:
        return 0
    starts = np.asarray(event_off[:-1], np.int64)
    starts = starts[(starts >= 0) & (starts < len(words))]
    return int((np.asarray(words)[starts].astype(np.uint32) & np.uint32(0xFFF)).astype(np.int64).sum())


@dataclass
class DeviceConstants:
    F: torch.Tensor
    q: torch.Tensor
    cfg: SvtConfig

    @classmethod
    def from_numpy(cls, F, q, cfg, device="cuda"):
        return cls(to_device_i16(F, device), to_device_i16(q, device), cfg)


class DevicePointer:
    """A raw device address with the `data_ptr()` the wrappers take."""

    def __init__(self, ptr: int):
        self.ptr = int(ptr)

    def data_ptr(self) -> int:
        return self.ptr


class MappedHost:
    """Pinned host memory mapped into the GPU's address space (svt_host_alloc):
    `host` is a numpy byte view for the CPU, `device(offset)` an address the
    kernels read and write in place."""

    def __init__(self, nbytes: int):
        h, d = ctypes.c_void_p(), ctypes.c_void_p()
        N.check(N.load().svt_host_alloc(int(nbytes), ctypes.byref(h), ctypes.byref(d)),
                "svt_host_alloc")
        self.nbytes = int(nbytes)
        self._h, self._d = h.value, d.value
        self.host = np.ctypeslib.as_array((ctypes.c_uint8 * self.nbytes).from_address(self._h))

    def view(self, dtype, offset: int = 0, count: int | None = None) -> np.ndarray:
        n = (self.nbytes - offset) // np.dtype(dtype).itemsize if count is None else count
        return self.host[offset: offset + n * np.dtype(dtype).itemsize].view(dtype)

    def device(self, offset: int = 0) -> DevicePointer:
        return DevicePointer(self._d + int(offset))

    def close(self):
        if self._h:
            self.host = None
            N.check(N.load().svt_host_free(ctypes.c_void_p(self._h)), "svt_host_free")
            self._h = self._d = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FusedPath:
    """Buffers of the fused path for batches up to the given capacities."""

    def __init__(self, max_words, max_events, road_cap, consts: DeviceConstants, sched=None,
                 device="cuda"):
        self.max_words, self.max_events, self.road_cap = int(max_words), int(max_events), int(road_cap)
        self.consts = consts
        self.sched = sched
        ws = svt_run_workspace_size(self.max_words, self.max_events, self.road_cap, sched)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=device)
        self.out = torch.empty(max(self.road_cap, 1) * 6, dtype=torch.int32, device=device)
        self.event_road = torch.empty(self.max_events + 1, dtype=torch.int32, device=device)
        self.counts = torch.zeros(4, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int64, device=device)

    def run(self, words, n_words, event_off, n_events, stream=None, timer=None):
        if n_words > self.max_words or n_events > self.max_events:
            raise N.SvtError("batch larger than the buffers")
        svt_run(words, n_words, event_off, n_events, self.consts.F, self.consts.q, self.consts.cfg,
                self.road_cap, self.out, self.event_road, self.counts, self.status, self.workspace,
                self.sched, timer, stream)

    def result(self):
        """(status key, records [R, 6] uint32, counts) -- synchronises."""
        status = int(u64(self.status)[0])
        counts = u64(self.counts).copy()
        R = int(counts[0])
        rec = u32(self.out[: min(R, self.road_cap) * 6]).reshape(-1, 6) if status == N.STATUS_OK else None
        return status, rec, counts


class GraphPath:
    """svt_graph_* over a FusedPath's buffers: the fused launch sequence
    captured once with the batch sizes read on the device, then replayed for
    every batch whose words and offsets sit in `words` / `event_off`."""

    def __init__(self, path: FusedPath, words, event_off):
        c = path.consts
        self.path = path
        self.sizes = torch.zeros(2, dtype=torch.int64, device=path.out.device)
        self._keep = (words, event_off)
        h = ctypes.c_void_p()
        N.check(N.load().svt_graph_create(
            _p(words), path.max_words, _p(event_off), path.max_events, _p(self.sizes), _p(c.F),
            _p(c.q), ctypes.byref(c.cfg), path.road_cap, _p(path.out), _p(path.event_road),
            _p(path.counts), _p(path.status), _p(path.workspace), path.workspace.numel(),
            ctypes.byref(path.sched) if path.sched is not None else None, ctypes.byref(h)),
            "svt_graph_create")
        self.handle = h

    def set_sizes(self, n_words: int, n_events: int):
        self.sizes.copy_(torch.tensor([int(n_words), int(n_events)], dtype=torch.int64))

    def launch(self, stream=None):
        N.check(N.load().svt_graph_launch(self.handle, _stream(stream)), "svt_graph_launch")

    def close(self):
        if getattr(self, "handle", None):
            N.load().svt_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class PlainPath:
    """Buffers of the plain per-stage path."""

    def __init__(self, max_words, max_events, road_cap, comb_cap, consts: DeviceConstants,
                 device="cuda"):
        self.max_words, self.max_events = int(max_words), int(max_events)
        self.road_cap, self.comb_cap = int(road_cap), int(comb_cap)
        self.consts = consts
        d = device
        rc, cc = max(self.road_cap, 1), max(self.comb_cap, 1)
        self.ws_unpack = torch.empty(svt_unpack_workspace_size(self.max_words), dtype=torch.uint8, device=d)
        self.ws_combine = torch.empty(svt_combine_workspace_size(self.road_cap), dtype=torch.uint8, device=d)
        self.road_word = torch.empty(rc, dtype=torch.int32, device=d)
        self.road_nhit = torch.empty(rc, dtype=torch.int32, device=d)
        self.event_road = torch.empty(self.max_events + 1, dtype=torch.int32, device=d)
        self.n_roads = torch.zeros(1, dtype=torch.int64, device=d)
        self.status = torch.zeros(1, dtype=torch.int64, device=d)
        self.road_flags = torch.empty(rc, dtype=torch.int32, device=d)
        self.comb_off = torch.empty(rc + 1, dtype=torch.int64, device=d)
        self.comb_road = torch.empty(cc, dtype=torch.int32, device=d)
        self.comb_hits = torch.empty(cc, dtype=torch.int32, device=d)
        self.n_combs = torch.zeros(1, dtype=torch.int64, device=d)
        self.fit_chi2 = torch.empty(cc, dtype=torch.int32, device=d)
        self.fit_par = torch.empty(3 * cc, dtype=torch.int32, device=d)
        self.best = torch.empty(rc * 6, dtype=torch.int32, device=d)
        self.out = torch.empty(rc * 6, dtype=torch.int32, device=d)

    def run(self, words, n_words, event_off, n_events, stream=None, fit_events=None,
            stage_marks=None):
        """All five stages.  fit_events = (start, end) torch events recorded
        around the fit stage; stage_marks = six torch events recorded before
        unpack and after unpack, combine, fit, select and format -- all on the
        same stream."""
        c = self.consts
        st = stream if stream is not None else torch.cuda.current_stream()

        def mark(i):
            if stage_marks is not None:
                stage_marks[i].record(st)

        mark(0)
        svt_unpack(words, n_words, event_off, n_events, c.cfg.n_sectors, self.road_cap,
                   self.road_word, self.road_nhit, self.event_road, self.n_roads, self.status,
                   self.ws_unpack, stream, c.cfg.xft_pairs)
        mark(1)
        svt_combine(self.road_nhit, self.n_roads, self.road_cap, c.cfg, self.comb_cap,
                    self.road_flags, self.comb_off, self.comb_road, self.comb_hits, self.n_combs,
                    self.status, self.ws_combine, stream)
        mark(2)
        if fit_events is not None:
            fit_events[0].record(st)
        svt_fit(words, self.road_word, self.road_nhit, self.comb_road, self.comb_hits,
                self.n_combs, self.comb_cap, c.F, c.q, c.cfg, self.fit_chi2, self.fit_par,
                self.status, stream)
        if fit_events is not None:
            fit_events[1].record(st)
        mark(3)
        svt_select(self.fit_chi2, self.fit_par, self.comb_cap, self.comb_off, self.road_flags,
                   self.n_roads, self.road_cap, c.cfg, self.best, self.status, stream)
        mark(4)
        svt_format(self.best, words, self.road_word, self.n_roads, self.road_cap, self.out,
                   self.status, stream)
        mark(5)

    def result(self):
        status = int(u64(self.status)[0])
        R = int(u64(self.n_roads)[0])
        rec = u32(self.out[: min(R, self.road_cap) * 6]).reshape(-1, 6) if status == N.STATUS_OK else None
        return status, rec, R


def svt_run_host_workspace_size(max_words, max_events, road_cap, sched=None) -> int:
    return N.load().svt_run_host_workspace_size(max_words, max_events, road_cap,
                                                ctypes.byref(sched) if sched is not None else None)


def svt_run_host(h_words, n_words, h_event_off, n_events, F, q, cfg, road_cap, h_out, h_status,
                 workspace, sched=None, stream=None) -> int:
    """svt_run_host: copy in, fused path, copy out, all on `stream`; returns
    the number of records that land in h_out (pinned host tensors)."""
    n = ctypes.c_uint64()
    N.check(N.load().svt_run_host(_p(h_words), n_words, _p(h_event_off), n_events, _p(F), _p(q),
                                  ctypes.byref(cfg), road_cap, _p(h_out), _p(h_status),
                                  ctypes.byref(n), _p(workspace), workspace.numel(),
                                  ctypes.byref(sched) if sched is not None else None,
                                  _stream(stream)), "svt_run_host")
    return int(n.value)


class StreamingRunner:
    """A stream of batches from pinned host memory through svt_run_host (copy
    in, fused path, copy out as one library call per batch).  `depth` sets of
    (CUDA stream, device workspace, pinned outputs) take the batches in turn,
    so one batch's copies overlap another's compute; each batch still carries
    its own H2D copy and D2H read.  A set's outputs are overwritten `depth`
    batches later."""

    def __init__(self, max_words, max_events, road_cap, consts: DeviceConstants, sched=None,
                 device="cuda", depth: int = 2):
        self.depth = int(depth)
        self.consts, self.sched = consts, sched
        self.max_words, self.max_events = int(max_words), int(max_events)
        self.road_cap = int(road_cap)
        ws = svt_run_host_workspace_size(self.max_words, self.max_events, self.road_cap, sched)
        self.workspace = [torch.empty(ws, dtype=torch.uint8, device=device)
                          for _ in range(self.depth)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(self.depth)]
        self.h_out = [torch.empty(max(self.road_cap, 1) * 6, dtype=torch.int32, pin_memory=True)
                      for _ in range(self.depth)]
        self.h_status = [torch.empty(1, dtype=torch.int64, pin_memory=True) for _ in range(self.depth)]
        self.n_out = [0] * self.depth
        self.i = 0

    def submit(self, h_words, h_event_off, n_roads=None, marks=None):
        """Enqueue one batch; `marks` = (start, end) torch events recorded on the
        batch's stream before its copy-in and after its copy-out.  Returns the
        bytes (h2d, d2h)."""
        k = self.i % self.depth
        n_words, n_events = h_words.numel(), h_event_off.numel() - 1
        if n_words > self.max_words or n_events > self.max_events:
            raise N.SvtError("batch larger than the buffers")
        st = self.streams[k]
        if marks is not None:
            marks[0].record(st)
        c = self.consts
        n_rec = svt_run_host(h_words, n_words, h_event_off, n_events, c.F, c.q, c.cfg,
                             self.road_cap, self.h_out[k], self.h_status[k], self.workspace[k],
                             self.sched, st)
        if marks is not None:
            marks[1].record(st)
        self.n_out[k] = n_rec
        self.i += 1
        return 4 * n_words + 8 * (n_events + 1), 24 * n_rec + 8

    def wait(self):
        """(status key, records [R, 6] uint32) of the last submitted batch."""
        for st in self.streams:
            st.synchronize()
        k = (self.i - 1) % self.depth
        return self.result(k)

    def result(self, k):
        """(status key, records) held by set k (after wait)."""
        status = int(self.h_status[k].numpy().view(np.uint64)[0])
        rec = self.h_out[k][: 6 * self.n_out[k]].numpy().view(np.uint32).reshape(-1, 6)
        return status, rec


FUSED_LAUNCHES_PER_RUN = 3   # prologue, unpack_roads (one pass over the tiles), fit
PLAIN_LAUNCHES_PER_RUN = 11  # unpack (3), combine (5), fit, select, format


class HostRunner:
    """End-to-end use from host memory: pinned host buffers, the H2D copy of a
    batch, the CUDA path on the device and the D2H copy of the records and
    the status, all enqueued on one stream.

    ``path`` is a FusedPath or a PlainPath sized for the largest batch.
    """

    def __init__(self, path, stream=None):
        self.path = path
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        dev = path.out.device
        self.d_words = torch.empty(max(path.max_words, 4), dtype=torch.int32, device=dev)
        self.d_event_off = torch.empty(path.max_events + 1, dtype=torch.int64, device=dev)
        self.h_out = torch.empty(path.out.numel(), dtype=torch.int32, pin_memory=True)
        self.h_status = torch.empty(1, dtype=torch.int64, pin_memory=True)
        self.n_roads = 0

    @staticmethod
    def pin_batch(words: np.ndarray, event_off: np.ndarray):
        """Pinned host copies of a batch (uint32 words, uint64 offsets)."""
        w = torch.from_numpy(np.ascontiguousarray(words, np.uint32).view(np.int32)).pin_memory()
        e = torch.from_numpy(np.ascontiguousarray(event_off, np.uint64).view(np.int64)).pin_memory()
        return w, e

    def submit(self, h_words, h_event_off, n_roads):
        """Enqueue H2D + run + D2H of one batch; returns the bytes moved (h2d, d2h)."""
        n_words, n_events = h_words.numel(), h_event_off.numel() - 1
        with torch.cuda.stream(self.stream):
            self.d_words[:n_words].copy_(h_words, non_blocking=True)
            self.d_event_off[: n_events + 1].copy_(h_event_off, non_blocking=True)
            self.path.run(self.d_words, n_words, self.d_event_off, n_events, stream=self.stream)
            n_out = min(n_roads, self.path.road_cap) * 6
            self.h_out[:n_out].copy_(self.path.out[:n_out], non_blocking=True)
            self.h_status.copy_(self.path.status, non_blocking=True)
        self.n_roads = n_roads
        return 4 * n_words + 8 * (n_events + 1), 4 * n_out + 8

    def wait(self):
        """(status key, records [R, 6] uint32) of the last submitted batch."""
        self.stream.synchronize()
        status = int(self.h_status.numpy().view(np.uint64)[0])
        n = min(self.n_roads, self.path.road_cap)
        rec = self.h_out[: n * 6].numpy().view(np.uint32).reshape(-1, 6)
        return status, rec
