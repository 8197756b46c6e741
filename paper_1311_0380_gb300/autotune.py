"""Schedule autotuning for the fused path: the timing loop runs natively
(svt_autotune in libsvt.so, CUDA events); this module keeps the chosen
schedules in a JSON cache keyed by GPU and workload shape."""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

from . import _native as N
from .api import SvtSchedule, _p, _stream

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "svt_gb300", "schedules.json")


def signature(n_words: int, n_events: int, road_cap: int, cfg, flushed: bool = False) -> str:
    """Workload key: GPU name, powers of two of the sizes, the fit config and
    whether the runs were timed with L2 flushed."""
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    b = lambda v: int(math.log2(max(int(v), 1)))
    return (f"{name}|w{b(n_words)}|e{b(n_events)}|r{b(road_cap)}|c{cfg.max_comb}|"
            f"m{cfg.min_layers}|s{cfg.n_sectors}|l{int(flushed)}")


def tune(path, words, n_words, event_off, n_events, reps: int = 3, flush=None):
    """Time every candidate schedule on this batch with `path` (a FusedPath)
    and return (SvtSchedule, mean ms).  `flush`: an optional device tensor
    larger than L2, overwritten before every timed run so that each run
    starts with none of the batch in L2."""
    best = SvtSchedule()
    ms = ctypes.c_float()
    c = path.consts
    fb = flush.numel() * flush.element_size() if flush is not None else 0
    N.check(N.load().svt_autotune(_p(words), n_words, _p(event_off), n_events, _p(c.F), _p(c.q),
                                  ctypes.byref(c.cfg), path.road_cap, _p(path.out),
                                  _p(path.status), _p(path.workspace), path.workspace.numel(), reps,
                                  _p(flush), fb,
                                  ctypes.byref(best), ctypes.byref(ms), _stream(None)),
            "svt_autotune")
    return best, float(ms.value)


def tuned_schedule(path, words, n_words, event_off, n_events, cache: str | None = DEFAULT_CACHE,
                   reps: int = 3, flush=None):
    """Cached schedule for this GPU and workload shape, tuning on a miss."""
    key = signature(n_words, n_events, path.road_cap, path.consts.cfg, flush is not None)
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if key in table:
        v = table[key]
        return SvtSchedule(v["warps_per_block"], v["blocks_per_sm"], v["rows_per_item"],
                           v["roads_per_chunk"], v["small_max"], v.get("pair_small", 0)), v.get("ms")
    sch, ms = tune(path, words, n_words, event_off, n_events, reps, flush)
    table[key] = {f: getattr(sch, f) for f, _ in SvtSchedule._fields_}
    table[key]["ms"] = ms
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return sch, ms
