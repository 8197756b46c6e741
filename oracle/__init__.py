"""CPU oracle of the SVT linearised track fit -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.

``svt_oracle.c`` is the integer path (unpack, combine, fit, cut, select,
format; the paper's Sec. 2 and Sec. 2.1), compiled with gcc into
``liborc.so`` and reached through ctypes.  ``calib.py`` is the FP64 reference of
the FP32 calibration relaxation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "svt_oracle.c")
LIB = os.path.join(HERE, "liborc.so")

KEY_OK = (1 << 64) - 1
E_BAD_ARG, E_BAD_TYPE, E_BAD_RESERVED, E_BAD_LAYER = 1, 2, 3, 4
E_UNSORTED, E_TOO_MANY_HITS, E_BAD_SECTOR, E_NROADS_MISMATCH = 5, 6, 7, 8
E_BAD_CONFIG = 10
E_XFT_UNPAIRED = 12
F_PASS, F_OVERFLOW, F_BAD_PATTERN, F_NO_HITS = 1, 2, 4, 8


class OrcConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("oshift", "qshift", "chi2_cut", "max_comb", "min_layers", "n_sectors",
                 "xft_pairs")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i16p = ctypes.POINTER(ctypes.c_int16)
            i64p = ctypes.POINTER(ctypes.c_int64)
            cfgp = ctypes.POINTER(OrcConfig)
            u64 = ctypes.c_uint64
            L.orc_validate.restype = u64
            L.orc_validate.argtypes = [u32p, u64, u64p, u64, ctypes.c_uint32, ctypes.c_uint32]
            L.orc_fit_one.restype = None
            L.orc_fit_one.argtypes = [i16p, i16p, u32p, ctypes.c_uint32, ctypes.c_uint32, i64p, u32p]
            L.orc_road.restype = u64
            L.orc_road.argtypes = [u32p, u32p, ctypes.c_uint32, ctypes.c_uint32, i16p, i16p, cfgp,
                                   u32p, u32p, i64p]
            for name in ("orc_run", "orc_run_omp"):
                f = getattr(L, name)
                f.restype = u64
                f.argtypes = [u32p, u64, u64p, u64, i16p, i16p, cfgp, u32p, u64, u64p]
            L.orc_run_roads.restype = None
            L.orc_run_roads.argtypes = [u32p, u64, u64p, u64, i16p, i16p, cfgp, u32p]
            L.orc_config_ok.restype = ctypes.c_int
            L.orc_config_ok.argtypes = [cfgp]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def config(oshift=15, qshift=15, chi2_cut=0xFFFFFFFF, max_comb=262144, min_layers=5, n_sectors=512,
           xft_pairs=0):
    return OrcConfig(oshift, qshift, chi2_cut, max_comb, min_layers, n_sectors, xft_pairs)


def validate(words, event_off, n_sectors, xft_pairs=0):
    words = np.ascontiguousarray(words, np.uint32)
    event_off = np.ascontiguousarray(event_off, np.uint64)
    return int(lib().orc_validate(_p(words, ctypes.c_uint32), len(words),
                                  _p(event_off, ctypes.c_uint64), len(event_off) - 1, n_sectors,
                                  xft_pairs))


def decode_key(key):
    """(word_index, code) of a status key, or None when it is the OK key."""
    if key == KEY_OK:
        return None
    return key >> 8, key & 0xFF


def fit_one(F36, q6, x6, oshift=15, qshift=15):
    F36 = np.ascontiguousarray(F36, np.int16).reshape(36)
    q6 = np.ascontiguousarray(q6, np.int16).reshape(6)
    x6 = np.ascontiguousarray(x6, np.uint32).reshape(6)
    y = np.zeros(6, np.int64)
    chi2 = np.zeros(1, np.uint32)
    lib().orc_fit_one(_p(F36, ctypes.c_int16), _p(q6, ctypes.c_int16), _p(x6, ctypes.c_uint32),
                      oshift, qshift, _p(y, ctypes.c_int64), _p(chi2, ctypes.c_uint32))
    return y, int(chi2[0])


def road(n, coords, sector, road_id, F, q, cfg, detail=False):
    """One road.  ``coords[l]`` lists the coordinates of layer l's hits.

    Returns (record[6], chi2 per combination, y per combination) when
    ``detail`` is set, else the record alone.
    """
    n = np.ascontiguousarray(n, np.uint32)
    buf = np.zeros((6, 16), np.uint32)
    for l in range(6):
        buf[l, : n[l]] = coords[l][: n[l]]
    F = np.ascontiguousarray(F, np.int16)
    q = np.ascontiguousarray(q, np.int16)
    rec = np.zeros(6, np.uint32)
    C = 1
    for l, v in enumerate(n):
        C *= 1 if (l == 5 and cfg.xft_pairs) else max(int(v), 1)
    n_eval = min(C, cfg.max_comb) if detail else 0
    all_chi2 = np.zeros(max(n_eval, 1), np.uint32)
    all_y = np.zeros((max(n_eval, 1), 6), np.int64)
    got = lib().orc_road(_p(n, ctypes.c_uint32), _p(buf, ctypes.c_uint32), sector, road_id,
                         _p(F, ctypes.c_int16), _p(q, ctypes.c_int16), ctypes.byref(cfg),
                         _p(rec, ctypes.c_uint32),
                         _p(all_chi2, ctypes.c_uint32) if detail else None,
                         _p(all_y, ctypes.c_int64) if detail else None)
    if detail:
        return rec, all_chi2[:got], all_y[:got]
    return rec


def run(words, event_off, F, q, cfg, omp=False):
    """Whole batch: returns (status_key, records [R, 6] uint32)."""
    words = np.ascontiguousarray(words, np.uint32)
    event_off = np.ascontiguousarray(event_off, np.uint64)
    F = np.ascontiguousarray(F, np.int16)
    q = np.ascontiguousarray(q, np.int16)
    n_events = len(event_off) - 1
    cap = max(len(words), 1)
    if n_events > 0 and len(words) > 0:
        # the event headers bound the road count once the batch is valid
        hdr = words[event_off[:-1].astype(np.int64).clip(0, len(words) - 1)]
        cap = int((hdr & 0xFFF).astype(np.int64).sum()) if len(hdr) else 0
    out = np.zeros((max(cap, 1), 6), np.uint32)
    n_roads = np.zeros(1, np.uint64)
    f = lib().orc_run_omp if omp else lib().orc_run
    key = int(f(_p(words, ctypes.c_uint32), len(words), _p(event_off, ctypes.c_uint64), n_events,
                _p(F, ctypes.c_int16), _p(q, ctypes.c_int16), ctypes.byref(cfg),
                _p(out, ctypes.c_uint32), cap, _p(n_roads, ctypes.c_uint64)))
    if key != KEY_OK:
        return key, None
    return key, out[: int(n_roads[0])]


def run_roads(words, road_pos, F, q, cfg):
    """Records of the roads whose header words sit at ``road_pos``."""
    words = np.ascontiguousarray(words, np.uint32)
    road_pos = np.ascontiguousarray(road_pos, np.uint64)
    F = np.ascontiguousarray(F, np.int16)
    q = np.ascontiguousarray(q, np.int16)
    out = np.zeros((max(len(road_pos), 1), 6), np.uint32)
    lib().orc_run_roads(_p(words, ctypes.c_uint32), len(words), _p(road_pos, ctypes.c_uint64),
                        len(road_pos), _p(F, ctypes.c_int16), _p(q, ctypes.c_int16),
                        ctypes.byref(cfg), _p(out, ctypes.c_uint32))
    return out[: len(road_pos)]


def num_threads():
    return int(lib().orc_num_threads())
