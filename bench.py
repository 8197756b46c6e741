#!/usr/bin/env python3
"""Benchmark of the SVT track-fit hot path on GB300.

One step = one batch of the scaled-up workload (3000 events; roads per event
Poisson(64); hits per layer geometric with mean 3 capped at 8; 512 sectors)
through unpack -> combine -> fit -> cut -> select -> format.  The fused
persistent path is the headline; the plain per-stage path is timed beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead: the paper ships no code, so the oracle is the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fits/sec"
UNIT = "fits/s"
# Algorithmic integer operations per fitted combination in the direct form of
# the fit: 36 multiply-adds, 6 offset adds, 6 shifts, 3 clamps, 3 squares,
# 2 adds and 1 compare.  The fused kernel shares partial sums between
# combinations and executes fewer, so its fraction of this peak can pass 1.
OPS_PER_FIT = 57
# int32 peak: 152 SMs x 128 int32 lanes (ALU and FMA pipes, 64 each) x 2.07 GHz
N_SM, LANES_PER_SM, SM_MAX_GHZ = 152, 128, 2.07
# plain-path fit kernel: 8 B of combination record read, 16 B of results written
PLAIN_BYTES_PER_FIT = 24
ALU_PEAK_TOPS = N_SM * LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
# instruction issue: 4 schedulers per SM, one warp instruction each per cycle
ISSUE_PEAK_GINST = N_SM * 4 * SM_MAX_GHZ
# the fit kernel and the road descriptors that shape its work
FIT_KERNEL_SRC = [os.path.join(ROOT, "paper_1311_0380_gb300", "csrc", f)
                  for f in ("svt_fused.cu", "svt_roads.cuh")]
TRAFFIC_NOTE = os.path.join(ROOT, "profiles", "fit_persistent_scaled3000.md")
UNEVEN_NOTE = os.path.join(ROOT, "profiles", "fit_persistent_uneven512.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="svt", choices=["svt", "reference"])
    ap.add_argument("--workload", default="scaled",
                    choices=["scaled", "paper", "uneven", "small", "xft"])
    ap.add_argument("--events", type=int, default=3000)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serve-short", action="store_true",
                    help="serve 30k and 100k events instead of 10 s at 30 kHz and 1M at 300 kHz")
    ap.add_argument("--no-calib", action="store_true", help="skip the FP32 calibration measurement")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the full-size uneven workload (65536 events per launch)")
    ap.add_argument("--no-batch-sweep", action="store_true",
                    help="skip the scaled workload's batch sizes (1, 10, 100, 1000, 3000 events)")
    ap.add_argument("--no-tune", action="store_true", help="use the default schedule")
    ap.add_argument("--sweep", action="store_true",
                    help="latency against the number of fits for the paper-shape workload "
                         "(Sec. 4.1): CPU oracle serial and per-event threads, fused and "
                         "plain paths, plain-path stage breakdown; prints one JSON line")
    ap.add_argument("--sweep-reps", type=int, default=100)
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--bps", type=int, default=0)
    ap.add_argument("--pair", action="store_true",
                    help="pair small roads on half warps (schedule field pair_small = 1)")
    ap.add_argument("--quad", action="store_true",
                    help="also group tiny roads four to a warp (pair_small = 2)")
    ap.add_argument("--lanes", action="store_true",
                    help="tiny roads on lanes of their own, 32 roads per chunk unless --chunk "
                         "says otherwise (pair_small = 3)")
    ap.add_argument("--chunk", type=int, default=0, help="roads per chunk of the schedule")
    return ap.parse_args()


def dist_setup(args, backend=None):
    """One process per GPU, as launched by torchrun: rank, world size and
    local rank come from the environment.  The reference arm runs on host
    cores only, so it joins over gloo."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            gpu = torch.cuda.is_available() and args.impl != "reference"
            backend = "nccl" if gpu else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def dist_teardown(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def reduce_over_ranks(world, ms, units, device="cpu"):
    """Whole-job figures: the slowest rank's time and the sum of every rank's
    units (each rank fits its own batch, so their fit counts differ)."""
    if world == 1:
        return float(ms), [int(u) for u in units]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([int(x) for x in units], dtype=torch.int64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), [int(x) for x in u.tolist()]


def file_sha(paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_profile(key, note=TRAFFIC_NOTE):
    """A figure of the fit kernel from a committed ncu summary (`key: value
    kernel_sha: sha`), or None when the summary is absent or the kernel source
    changed since."""
    try:
        text = open(note).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.eE+]+)\s+kernel_sha:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != file_sha(FIT_KERNEL_SRC):
        return None
    return float(m.group(1))


def recorded_traffic():
    """Per-launch DRAM bytes of the fit kernel (ncu, full-size launch)."""
    return recorded_profile("traffic_bytes_per_launch")


def recorded_schedule(note=TRAFFIC_NOTE):
    """The schedule the committed ncu figures were taken with
    (`profiled_schedule: field=value ... kernel_sha: sha`), or None."""
    try:
        text = open(note).read()
    except OSError:
        return None
    m = re.search(r"profiled_schedule:\s*((?:\w+=\d+\s+)+)kernel_sha:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != file_sha(FIT_KERNEL_SRC):
        return None
    return {k: int(v) for k, v in (kv.split("=") for kv in m.group(1).split())}


def same_work_split(a, b, max_comb):
    """Whether two schedules give the fit kernel the same work units, so that
    its instructions per combination agree: the same roads per chunk and
    grouping, and -- where roads are split at all (small_max below the
    workload's cap) -- the same split threshold and rows per item."""
    if a is None or b is None:
        return False
    defaults = {"warps_per_block": 8, "rows_per_item": 16, "roads_per_chunk": 4,
                "small_max": 4096}   # what zero fields of a schedule mean

    def key(s):
        s = {f: (v or defaults.get(f, v)) for f, v in s.items()}
        split = s["small_max"] < max_comb
        return (s["roads_per_chunk"], s["pair_small"], s["rows_per_item"] if split else None,
                s["small_max"] if split else None)
    return key(a) == key(b)


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="svt_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


TILE_DRAW = 4096   # batches larger than this many events repeat one draw of it


def workload(args, rank):
    from paper_1311_0380_gb300 import synth
    spec = synth.SPECS[args.workload]
    consts = synth.make_constants(spec.n_sectors)
    # every rank fits its own batch (independent events): weak scaling
    seed = spec.seed + 7919 * rank
    if args.events > TILE_DRAW and args.events % TILE_DRAW == 0:
        batch = synth.tile_batch(synth.make_batch(spec, TILE_DRAW, consts, seed=seed),
                                 args.events // TILE_DRAW)
    else:
        batch = synth.make_batch(spec, args.events, consts, seed=seed)
    return spec, consts, batch


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0   # fallback figure of the profiling recipe


def percentile(xs, p):
    return float(np.percentile(np.asarray(xs, np.float64), p)) if xs else None


def cpu_baseline(spec, consts, batch, budget_s=12.0):
    """The oracle as it stands (serial C), on a bounded sample of the batch."""
    import oracle
    cfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors,
                        int(spec.xft))
    fits_ev = batch.combinations(spec.max_comb)
    # event prefix sized for about budget_s of serial work (~12 Mfits/s per core)
    road_end = np.cumsum(batch.n_roads)
    fits_cum = np.concatenate([[0], np.cumsum(fits_ev)])
    target = budget_s * 12e6
    n_ev = int(np.searchsorted(fits_cum[road_end], target)) + 1
    n_ev = max(1, min(n_ev, batch.n_events))
    n_words = int(batch.event_off[n_ev])
    words = batch.words[:n_words]
    off = batch.event_off[: n_ev + 1]
    fits = int(fits_cum[road_end[n_ev - 1]])
    t0 = time.perf_counter()
    key, _ = oracle.run(words, off, consts.F, consts.q, cfg, omp=False)
    dt = time.perf_counter() - t0
    assert key == oracle.KEY_OK
    return {"value": fits / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_ev} of {batch.n_events} events ({fits} fits), serial C oracle, one pass",
            "seconds": round(dt, 3)}


def cpu_baseline_omp(spec, consts, batch):
    """The same oracle with one event per OpenMP thread on every host core
    (how the paper ran the event loop on the many-core coprocessor), over the
    whole batch."""
    import oracle
    cfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors,
                        int(spec.xft))
    fits = int(batch.combinations(spec.max_comb).sum())
    oracle.run(batch.words[: int(batch.event_off[min(50, batch.n_events)])],
               batch.event_off[: min(50, batch.n_events) + 1], consts.F, consts.q, cfg, omp=True)
    t0 = time.perf_counter()
    key, _ = oracle.run(batch.words, batch.event_off, consts.F, consts.q, cfg, omp=True)
    dt = time.perf_counter() - t0
    assert key == oracle.KEY_OK
    return {"value": fits / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "nproc": os.cpu_count(), "kind": "oracle",
            "sample": f"all {batch.n_events} events ({fits} fits), C oracle, one event per "
                      "OpenMP thread, one pass",
            "seconds": round(dt, 3)}


CALIB_TRACKS = 1 << 20


def calibration(dev, reps=20):
    """The calibration section of the bench line: the workload's 1M tracks,
    and a 16M-track batch beside it (large-batch bandwidth)."""
    out = calibration_one(dev, CALIB_TRACKS, reps)
    out["large_batch"] = calibration_one(dev, 16 * CALIB_TRACKS, reps)
    return out


def calibration_one(dev, n_tracks, reps):
    """The FP32 relaxation on n_tracks generated tracks over 512 sectors: the
    forward y = F[s] x + q[s], the loss alone, the loss and its gradient in
    one fused pass (what autograd runs), the scaling of that gradient by the
    upstream one, and the separate backward pass (svt_calib_loss_backward),
    each timed with CUDA events over `reps` calls with the L2 flushed (by a
    256 MB read) before each, every call replayed from a one-call CUDA graph.
    Algorithmic bytes per track: the forward reads x (24 B) and writes y
    (24 B); the loss, the fused pass and the backward read x and the true
    parameters (36 B)."""
    import torch
    from paper_1311_0380_gb300 import calib, synth
    consts = synth.make_constants(512)
    cs = synth.make_calib(n_tracks, consts)
    data = calib.CalibData(cs.x, cs.sector, cs.theta, 512, cs.weight, device=dev)
    F = torch.tensor(cs.F0, dtype=torch.float32, device=dev, requires_grad=True)
    q = torch.tensor(cs.q0, dtype=torch.float32, device=dev, requires_grad=True)
    # L2 flush by reading 256 MB (the lines it leaves are clean, so the timed
    # kernel pays no write-back of the flush's own data)
    flush_src = torch.ones(64 << 20, dtype=torch.int32, device=dev)
    flush_dst = torch.empty((), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    peak = measured_hbm_peak()

    def timed(fn):
        # one call captured in a CUDA graph and replayed right after the L2
        # flush, so host-side call overhead cannot stretch the device time
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                fn()
        stream.wait_stream(side)
        ms = []
        for i in range(reps):
            torch.sum(flush_src, 0, out=flush_dst)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    class _Ctx:   # what the autograd Functions keep between forward and backward
        def save_for_backward(self, *t):
            self.saved_tensors = t

        def mark_non_differentiable(self, *t):
            pass

    ctx_f, ctx_l, ctx_g, ctx_u = _Ctx(), _Ctx(), _Ctx(), _Ctx()
    ctx_l.needs_input_grad = (False, False, False)   # the loss alone
    ctx_g.needs_input_grad = (True, True, False)     # the loss and its gradient in one pass
    g1 = torch.ones((), device=dev)
    with torch.no_grad():
        t_fwd = timed(lambda: calib.FitFP32.forward(ctx_f, F, q, data))
        t_loss = timed(lambda: calib.CalibLoss.forward(ctx_l, F, q, data))
        t_lg = timed(lambda: calib.CalibLoss.forward(ctx_g, F, q, data))
        ctx_y = _Ctx()
        t_lgy = timed(lambda: calib.CalibLossFit.forward(ctx_y, F, q, data))
        t_scale = timed(lambda: calib.CalibLoss.backward(ctx_g, g1))
        calib.CalibLossUnfused.forward(ctx_u, F, q, data)
        t_bwd = timed(lambda: calib.CalibLossUnfused.backward(ctx_u, g1))
    loss = calib.calib_loss(F, q, data)
    n = n_tracks
    out = {"tracks": n, "sectors": 512, "loss_value": float(loss.item()), "peak_gbs": peak,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    for name, ms, bpt in (("forward", t_fwd, 48), ("loss", t_loss, 36),
                          ("loss_and_grad", t_lg, 36), ("loss_backward", t_bwd, 36)):
        gbs = n * bpt / (ms / 1e3) / 1e9
        out[name] = {"us": ms * 1e3, "bytes_per_track": bpt, "achieved_gbs": gbs,
                     "frac": gbs / peak, "tracks_per_s": n / (ms / 1e3)}
    out["grad_scale_us"] = t_scale * 1e3
    gbs = n * 60 / (t_lgy / 1e3) / 1e9
    out["loss_grad_and_fit"] = {"us": t_lgy * 1e3, "bytes_per_track": 60, "achieved_gbs": gbs,
                                "frac": gbs / peak}
    # a calibration step from one pass: the fitted parameters, the loss and
    # its gradient (x and theta read, y written: 60 B per track), then the
    # scaling by the upstream gradient
    ms = t_lgy + t_scale
    gbs = n * 60 / (ms / 1e3) / 1e9
    out["step_one_pass"] = {"us": ms * 1e3, "bytes_per_track": 60, "achieved_gbs": gbs,
                            "frac": gbs / peak}
    # a calibration step as the autograd graph runs it, with the fitted
    # parameters also produced: forward y, the fused loss and gradient, and
    # the scaling by the upstream gradient (84 algorithmic bytes per track)
    ms = t_fwd + t_lg + t_scale
    gbs = n * 84 / (ms / 1e3) / 1e9
    out["step_forward_loss_grad"] = {"us": ms * 1e3, "bytes_per_track": 84, "achieved_gbs": gbs,
                                     "frac": gbs / peak}
    return out


def serving(dev, short=False):
    """Poisson arrivals of events shaped like the uneven workload (roads
    log-uniform in 1..2048, 1-16 hits per layer, 4096 combinations per road at
    most) at 30 kHz and 300 kHz through the continuous-batching server
    (fused path, 4 slots, CUDA graphs), and the plain per-stage path served one
    batch at a time at the same two rates beside it.  Latency = scheduled
    arrival to delivery of the event's result, H2D and D2H included.  The fused
    server runs 10 s or 1M events per rate, whichever comes first (300,000
    events at 30 kHz, 1,000,000 at 300 kHz; `short` runs 30,000 and 100,000);
    the plain server 30,000 events per rate.  Every row carries the server's
    queue and batching counters and, from a host-side trace of every batch,
    the longest wait of a batch's first event before dispatch; a further
    300 kHz run with device timestamps gives the fraction of batches whose
    device work overlaps another slot's."""
    from paper_1311_0380_gb300 import api, serve, synth
    consts = synth.make_constants(512)
    pool_b = synth.make_batch("uneven", 1024, consts, seed=synth.BASE_SEED + 4)
    fits_ev = np.bincount(np.repeat(np.arange(pool_b.n_events), pool_b.n_roads),
                          weights=pool_b.combinations(4096), minlength=pool_b.n_events)
    pool = serve.pinned_pool(pool_b.words)
    cfg = api.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg, dev)
    out = {"events": "uneven-shaped, pool of 1024 distinct events cycled",
           "mean_words_per_event": float(len(pool_b.words) / pool_b.n_events),
           "mean_fits_per_event": float(fits_ev.mean()),
           "latency": "from each event's scheduled Poisson arrival to the delivery of its result"}

    def run(srv, rate, n, device_times=False):
        srv.reset_stats()
        srv.trace_start(1 << 21, device_times=device_times)
        lat, wall = srv.bench_poisson(pool, pool_b.event_off, rate, n, seed=7)
        tr = srv.trace_stop()
        st = srv.stats()
        ok = lat != np.uint64(2 ** 64 - 1)
        us = lat[ok].astype(np.float64) / 1e3
        reps, rest = divmod(n, pool_b.n_events)
        fits = float(reps * fits_ev.sum() + fits_ev[:rest].sum())
        nb = max(int(st["batches"]), 1)
        row = {"rate_hz": rate, "events": n, "failed": int((~ok).sum()),
               "p50_us": float(np.percentile(us, 50)), "p99_us": float(np.percentile(us, 99)),
               "p999_us": float(np.percentile(us, 99.9)), "max_us": float(us.max()),
               "events_per_s": n / wall, "fits_per_s": fits / wall, "wall_s": wall,
               "kept_up": bool(n / wall >= 0.99 * rate),
               "batches": int(st["batches"]), "events_per_batch": n / nb,
               "max_batch_events": int(st["max_batch_events"]),
               "max_queue_depth": int(st["max_queued"]),
               "dispatch_us_per_batch": st["launch_ns"] / 1e3 / nb,
               "deliver_us_per_batch": st["finish_ns"] / 1e3 / nb,
               "events_over_1ms": int((us > 1000).sum())}
        if len(tr):
            wait = (tr["t_dispatch_ns"] - tr["t_first_arrive_ns"]) / 1e3
            k = int(np.argmax(wait))
            row["longest_wait_us"] = float(wait[k])
            row["longest_wait_at_s"] = float((tr["t_dispatch_ns"][k] - tr["t_dispatch_ns"][0]) / 1e9)
            row["queue_after_dispatch_max"] = int(tr["queued_after"].max())
            if device_times:
                dev_us = tr["dev_end_us"] - tr["dev_start_us"]
                row["overlap_fraction"] = serve.overlap_fraction(tr)
                row["device_us_per_batch_p50"] = float(np.percentile(dev_us, 50))
        return row

    # one road per chunk of the fit's work queue; batches of up to four events
    # replay a second graph with one persistent block per SM
    sched = api.schedule(8, 0, 16, 1, 4096, 0)
    srv = serve.Server(dc, n_slots=4, max_words=1 << 22, max_events=256, max_roads=1 << 17,
                       sched=sched, small_batch_events=4, small_blocks_per_sm=1)
    out["fused_schedule"] = dict({f: getattr(sched, f) for f, _ in api.SvtSchedule._fields_},
                                 small_batch_events=4, small_blocks_per_sm=1)
    n30, n300 = (30000, 100000) if short else (300000, 1000000)
    run(srv, 30e3, 3000)   # warm-up
    out["fused_graph_4slots"] = [run(srv, 30e3, n30), run(srv, 300e3, n300)]
    out["fused_300khz_device_trace"] = run(srv, 300e3, 100000, device_times=True)
    srv.close()
    # the plain per-stage path, one batch in flight at a time
    plain = serve.Server(dc, n_slots=1, max_words=1 << 22, max_events=256, max_roads=1 << 17,
                         mode=1, max_combs=(1 << 17) * 4096)
    run(plain, 30e3, 300)   # warm-up
    out["plain_per_batch"] = [run(plain, 30e3, 30000), run(plain, 300e3, 30000)]
    plain.close()
    return out


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle, timed step by step on a bounded sample."""
    if rank != 0:
        return
    import oracle
    spec, consts, batch = workload(args, 0)
    cfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors,
                        int(spec.xft))
    # each step: a 30-event slice of the workload (about 1.1M fits for 'scaled')
    step_events = max(1, min(30, batch.n_events))
    ev_of_road = np.repeat(np.arange(batch.n_events), batch.n_roads)
    fits_ev = np.bincount(ev_of_road, weights=batch.combinations(spec.max_comb),
                          minlength=batch.n_events).astype(np.int64)
    slices = []
    for s in range(args.warmup + args.steps):
        e0 = (s * step_events) % max(1, batch.n_events - step_events + 1)
        e1 = e0 + step_events
        w0, w1 = int(batch.event_off[e0]), int(batch.event_off[e1])
        slices.append((batch.words[w0:w1], (batch.event_off[e0:e1 + 1] - batch.event_off[e0]),
                       int(fits_ev[e0:e1].sum())))
    for s in range(args.warmup):
        oracle.run(slices[s][0], slices[s][1], consts.F, consts.q, cfg)
    t0 = time.perf_counter()
    fits = 0
    for s in range(args.warmup, args.warmup + args.steps):
        key, _ = oracle.run(slices[s][0], slices[s][1], consts.F, consts.q, cfg)
        assert key == oracle.KEY_OK
        fits += slices[s][2]
    dt = time.perf_counter() - t0
    value = fits / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        # the same workload as the GPU arm's line (its batch, its fits per
        # batch); every timed step processes a sample of it
        "config": {"workload": f"{args.workload}-{batch.n_events}ev", "events": batch.n_events,
                   "roads": int(batch.total_roads),
                   "fits_per_step": int(fits_ev.sum()), "sectors": spec.n_sectors,
                   "max_comb": spec.max_comb,
                   "sample_events_per_step": step_events,
                   "sample_fits_per_step": fits / args.steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{step_events}-event slices of the {args.workload} workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


SWEEP_EVENTS = (1, 2, 5, 10, 20, 50, 100, 200, 500, 1000, 2000, 3000)


def run_sweep(args):
    """The shape of the paper's Sec. 4.1 on GB300: events of 2048
    combinations (32 roads x 2^6), 1 to 3000 events per batch, every batch
    processed `--sweep-reps` times.  Per batch size: the CPU oracle serial and
    with one event per thread (the paper's embarrassingly parallel strategy),
    the fused path with inputs resident and end to end from pinned host
    memory, and the plain per-stage path with the fraction of its time in
    unpack, combine, fit and select + format (the paper's breakdown)."""
    import torch
    import oracle
    from paper_1311_0380_gb300 import api, synth
    dev = torch.device("cuda", 0)
    spec = synth.SPECS["paper"]
    consts = synth.make_constants(spec.n_sectors)
    full = synth.make_batch(spec, max(SWEEP_EVENTS), consts)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors)
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors)
    dconst = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg, dev)
    stream = torch.cuda.current_stream()
    reps = max(3, args.sweep_reps)
    from paper_1311_0380_gb300 import autotune

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    rows = []
    for n_ev in SWEEP_EVENTS:
        n_words = int(full.event_off[n_ev])
        words, off = full.words[:n_words], full.event_off[: n_ev + 1].copy()
        R = int(np.sum(full.n_roads[:n_ev]))
        fits = int(np.sum(full.combinations(spec.max_comb)[:R]))
        d_words, d_off = api.to_device_u32(words, dev), api.to_device_u64(off, dev)
        # fused, resident, in the schedule the autotuner picks for this batch
        # (every road of this shape is small and alike: it pairs them on half
        # warps, and small batches keep fewer blocks resident)
        fp = api.FusedPath(n_words, n_ev, R, dconst, None, dev)
        sched, _ = autotune.tuned_schedule(fp, d_words, n_words, d_off, n_ev, cache=None, reps=2)
        fp.sched = sched
        for _ in range(3):
            fp.run(d_words, n_words, d_off, n_ev)
        evs = [ev_pair() for _ in range(reps)]
        for a, b in evs:
            a.record(stream)
            fp.run(d_words, n_words, d_off, n_ev)
            b.record(stream)
        torch.cuda.synchronize()
        st, rec, _ = fp.result()
        assert st == api.N.STATUS_OK
        fused = [a.elapsed_time(b) * 1e3 for a, b in evs]
        # fused, end to end through the library's one call (svt_run_host:
        # copy-in, the fused path and copy-out enqueued by one C call), one
        # batch in flight, timed from before its copy-in to after its copy-out
        runner = api.StreamingRunner(n_words, n_ev, R, dconst, sched, dev, depth=1)
        h_w, h_o = api.HostRunner.pin_batch(words, off)
        for _ in range(3):
            runner.submit(h_w, h_o)
            runner.wait()
        e2e = []
        for _ in range(reps):
            a, b = ev_pair()
            runner.submit(h_w, h_o, marks=(a, b))
            zst_e2e, rec_e2e = runner.wait()
            e2e.append(a.elapsed_time(b) * 1e3)
        assert zst_e2e == api.N.STATUS_OK and np.array_equal(rec_e2e, rec)
        # zero-copy: words and offsets stay in mapped host memory and the
        # kernels read them in place (the records go to device memory and are
        # copied back, or are written straight into host memory; the status
        # word is copied back either way)
        w_bytes = (4 * n_words + 255) // 256 * 256
        mh = api.MappedHost(w_bytes + 8 * (n_ev + 1) + 24 * max(R, 1))
        mh.view(np.uint32, 0, n_words)[:] = words
        mh.view(np.uint64, w_bytes, n_ev + 1)[:] = off
        out_off = w_bytes + 8 * (n_ev + 1)
        h_out = torch.empty(6 * max(R, 1), dtype=torch.int32, pin_memory=True)
        h_status = torch.empty(1, dtype=torch.int64, pin_memory=True)
        zc = {}
        for out_host in (False, True):
            def zc_step():
                out = mh.device(out_off) if out_host else fp.out
                api.svt_run(mh.device(0), n_words, mh.device(w_bytes), n_ev, dconst.F, dconst.q,
                            cfg, R, out, fp.event_road, fp.counts, fp.status, fp.workspace,
                            sched=sched)
                if not out_host:
                    h_out[: 6 * R].copy_(fp.out[: 6 * R], non_blocking=True)
                h_status.copy_(fp.status, non_blocking=True)
            for _ in range(3):
                zc_step()
            torch.cuda.synchronize()
            lat = []
            for _ in range(reps):
                a, b = ev_pair()
                a.record(stream)
                zc_step()
                b.record(stream)
                b.synchronize()
                lat.append(a.elapsed_time(b) * 1e3)
            got = (mh.view(np.uint32, out_off, 6 * R) if out_host else h_out[: 6 * R].numpy().view(np.uint32))
            zst = int(h_status.numpy().view(np.uint64)[0])
            assert zst == api.N.STATUS_OK and np.array_equal(got.reshape(-1, 6), rec)
            zc["zero_copy_in_out_us" if out_host else "zero_copy_in_us"] = statistics.mean(lat)
        mh.close()
        # plain per-stage path with its breakdown
        pp = api.PlainPath(n_words, n_ev, R, fits, dconst, dev)
        for _ in range(3):
            pp.run(d_words, n_words, d_off, n_ev)
        marks = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(reps)]
        for m in marks:
            pp.run(d_words, n_words, d_off, n_ev, stage_marks=m)
        torch.cuda.synchronize()
        pst, prec, _ = pp.result()
        assert pst == api.N.STATUS_OK and np.array_equal(prec, rec)
        stages = np.array([[m[i].elapsed_time(m[i + 1]) * 1e3 for i in range(5)] for m in marks])
        plain = stages.sum(1)
        frac = stages.sum(0) / stages.sum()
        # CPU oracle: serial, and one event per thread
        cpu_reps = max(1, min(reps, int(4e6 // fits)))
        t = []
        for _ in range(cpu_reps):
            t0 = time.perf_counter()
            key, orec = oracle.run(words, off, consts.F, consts.q, ocfg, omp=False)
            t.append((time.perf_counter() - t0) * 1e6)
        assert key == oracle.KEY_OK and np.array_equal(orec, rec)
        t_omp = []
        for _ in range(cpu_reps):
            t0 = time.perf_counter()
            oracle.run(words, off, consts.F, consts.q, ocfg, omp=True)
            t_omp.append((time.perf_counter() - t0) * 1e6)
        row = {"events": n_ev, "fits": fits,
               "cpu_serial_us": statistics.mean(t), "cpu_threads_us": statistics.mean(t_omp),
               "fused_us": statistics.mean(fused), "fused_p50_us": percentile(fused, 50),
               "fused_e2e_us": statistics.mean(e2e), **zc, "plain_us": float(plain.mean()),
               "plain_breakdown": {"unpack": float(frac[0]), "combine": float(frac[1]),
                                   "fit": float(frac[2]), "select_format": float(frac[3] + frac[4])},
               "cpu_reps": cpu_reps, "gpu_reps": reps,
               "fused_schedule": {f: getattr(sched, f) for f, _ in api.SvtSchedule._fields_}}
        row["speedup_fused_e2e_vs_serial"] = row["cpu_serial_us"] / row["fused_e2e_us"]
        row["speedup_fused_vs_serial"] = row["cpu_serial_us"] / row["fused_us"]
        rows.append(row)
        print(f"{n_ev:5d} ev {fits:8d} fits  serial {row['cpu_serial_us']:10.1f} us  "
              f"threads {row['cpu_threads_us']:9.1f}  fused {row['fused_us']:7.1f}  "
              f"e2e {row['fused_e2e_us']:7.1f}  zc {zc['zero_copy_in_us']:7.1f} "
              f"{zc['zero_copy_in_out_us']:7.1f}  plain {row['plain_us']:8.1f}  "
              f"[unpack {frac[0]:.2f} combine {frac[1]:.2f} fit {frac[2]:.2f}]",
              file=sys.stderr, flush=True)
        del fp, pp, runner
    print(json.dumps({"sweep": "paper-shape (2048 fits per event)", "cpu_threads": oracle.num_threads(),
                      "fused_schedule": "autotuned per batch size (in each row)",
                      "rows": rows}))


E2E_POOL_SLICES = 10


def end_to_end(args, spec, consts, dconst, sched, rank, world, dev, barrier):
    """Steps through the public API from pinned host memory: every step copies
    its own batch in (words and offsets) and reads its records and status
    back; the streaming runner overlaps step i's compute with step i+1's
    copy-in and step i-1's copy-out.  The steps cycle through E2E_POOL_SLICES
    distinct batches of the workload (a pool larger than the 129 MB L2), so
    no step finds its inputs cached from an earlier one.  At least 100 steps
    are timed (about 25 ms at 3000 events), so that one late host-side
    submission cannot stand for the whole run."""
    import torch
    from paper_1311_0380_gb300 import api, synth
    n_ev = args.events
    pool = synth.make_batch(spec, n_ev * E2E_POOL_SLICES, consts,
                            seed=spec.seed + 104729 + 7919 * rank)
    h_pool = torch.from_numpy(pool.words.view(np.int32)).pin_memory()
    road_end = np.concatenate([[0], np.cumsum(pool.n_roads)])
    fits_road = np.concatenate([[0], np.cumsum(pool.combinations(spec.max_comb))])
    slices = []
    for k in range(E2E_POOL_SLICES):
        e0, e1 = k * n_ev, (k + 1) * n_ev
        w0, w1 = int(pool.event_off[e0]), int(pool.event_off[e1])
        off = torch.from_numpy((pool.event_off[e0:e1 + 1] - pool.event_off[e0]).astype(np.int64))
        r0, r1 = int(road_end[e0]), int(road_end[e1])
        slices.append((h_pool[w0:w1], off.pin_memory(), r1 - r0, int(fits_road[r1] - fits_road[r0])))
    max_words = max(sl[0].numel() for sl in slices)
    road_cap = max(sl[2] for sl in slices)
    runner = api.StreamingRunner(max_words, n_ev, road_cap, dconst, sched, dev)
    for i in range(args.warmup):
        sl = slices[i % E2E_POOL_SLICES]
        runner.submit(sl[0], sl[1], sl[2])
    runner.wait()
    steps = max(args.steps, 100)
    marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(steps)]
    fits = h2d = d2h = 0
    used = []
    barrier()
    for i in range(steps):
        k = (args.warmup + i) % E2E_POOL_SLICES
        sl = slices[k]
        bi, bo = runner.submit(sl[0], sl[1], sl[2], marks=marks[i])
        fits += sl[3]
        h2d += bi
        d2h += bo
        used.append(k)
    st, rec = runner.wait()
    barrier()
    assert st == api.N.STATUS_OK and len(rec) == slices[used[-1]][2]
    total_ms = marks[0][0].elapsed_time(marks[-1][1])
    lat = [a.elapsed_time(b) * 1e3 for a, b in marks]
    job_ms, (job_fits,) = reduce_over_ranks(world, total_ms, [fits], dev)
    return {"value": job_fits / (job_ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d // steps), "d2h_bytes_per_step": int(d2h // steps),
            "p50_us": percentile(lat, 50), "p99_us": percentile(lat, 99),
            "inputs": f"svt_run_host (C entry: H2D, fused path, D2H on one stream) on two "
                      f"alternating streams; {E2E_POOL_SLICES} distinct {n_ev}-event batches "
                      f"({4 * h_pool.numel() / 1e6:.0f} MB) cycled from pinned host memory, each "
                      "step copying its own batch in and its records and status out",
            "ms_per_step": job_ms / steps, "steps": steps}


UNEVEN_EVENTS = 65536


SCALED_BATCH_SIZES = (1, 10, 100, 1000, 3000)
PAPER_BATCH_SIZES = (1, 100, 1000, 3000)


def batch_size_sweep(spec, batch, dconst, dev, flush, sizes=SCALED_BATCH_SIZES,
                     label="scaled, first N events of the headline batch", reps=20, warmup=3):
    """A workload's batch sizes (the first N events of one batch; for the
    scaled workload 1, 10, 100, 1000 and all 3000 events of the headline
    batch, for the paper's shape 1, 100, 1000 and 3000), each with the schedule the autotuner
    picks for it, the fused path beside the plain per-stage path, L2
    overwritten before every timed run.  Per size: latency with inputs
    resident in HBM (both paths), and end to end from pinned host memory,
    each run copying its batch in and its records and status back: the fused
    path through its one C call (svt_run_host), and both paths through the
    same Python runner (torch copies around the path's calls), so that the
    fused-vs-plain comparison carries the same host overhead on both sides.
    Every size checks that both paths give the same records."""
    import torch
    from paper_1311_0380_gb300 import api, autotune
    stream = torch.cuda.current_stream()
    road_end = np.concatenate([[0], np.cumsum(batch.n_roads)])
    fits_road = np.concatenate([[0], np.cumsum(batch.combinations(spec.max_comb))])

    def stats(us):
        return {"mean": statistics.mean(us), "p50": percentile(us, 50), "p99": percentile(us, 99)}

    def timed(run, on=None):
        """Latency (us) of `reps` runs, each after an L2 overwrite; events on
        the stream `on` (default: the current one)."""
        st = on if on is not None else stream
        for _ in range(warmup):
            run(None)
        torch.cuda.synchronize()
        us = []
        for i in range(reps):
            flush.fill_(i)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            run((a, b, st))
            b.synchronize()
            us.append(a.elapsed_time(b) * 1e3)
        return us

    rows = []
    for n_ev in sizes:
        n_words = int(batch.event_off[n_ev])
        words, off = batch.words[:n_words], batch.event_off[: n_ev + 1].copy()
        R = int(road_end[n_ev])
        fits = int(fits_road[R])
        d_w, d_o = api.to_device_u32(words, dev), api.to_device_u64(off, dev)
        fp = api.FusedPath(n_words, n_ev, R, dconst, None, dev)
        sched, _ = autotune.tuned_schedule(fp, d_w, n_words, d_o, n_ev, cache=None, flush=flush,
                                           reps=2)
        fp.sched = sched

        def fused_run(m):
            if m:
                m[0].record(m[2])
            fp.run(d_w, n_words, d_o, n_ev)
            if m:
                m[1].record(m[2])
        fused_us = timed(fused_run)
        fst, frec, _ = fp.result()
        pp = api.PlainPath(n_words, n_ev, R, fits, dconst, dev)

        def plain_run(m):
            if m:
                m[0].record(m[2])
            pp.run(d_w, n_words, d_o, n_ev)
            if m:
                m[1].record(m[2])
        plain_us = timed(plain_run)
        pst, prec, _ = pp.result()
        assert fst == api.N.STATUS_OK and pst == api.N.STATUS_OK and np.array_equal(frec, prec), \
            f"fused and plain paths differ at {n_ev} events"
        # end to end
        h_w, h_o = api.HostRunner.pin_batch(words, off)
        sr = api.StreamingRunner(n_words, n_ev, R, dconst, sched, dev, depth=1)

        def c_entry(m):
            sr.submit(h_w, h_o, marks=(m[0], m[1]) if m else None)
            sr.wait()
        e2e_us = timed(c_entry, sr.streams[0])
        est, erec = sr.wait()
        assert est == api.N.STATUS_OK and np.array_equal(erec, frec)
        py = {}
        for name, path in (("fused", fp), ("plain", pp)):
            hr = api.HostRunner(path, stream)

            def py_run(m, hr=hr):
                if m:
                    m[0].record(m[2])
                hr.submit(h_w, h_o, R)
                if m:
                    m[1].record(m[2])
                hr.wait()
            py[name] = timed(py_run)
            pst2, prec2 = hr.wait()
            assert pst2 == api.N.STATUS_OK and np.array_equal(prec2, frec)
        rows.append({
            "events": n_ev, "roads": R, "fits": fits,
            "h2d_bytes": 4 * n_words + 8 * (n_ev + 1), "d2h_bytes": 24 * R + 8,
            "schedule": {f: getattr(sched, f) for f, _ in api.SvtSchedule._fields_},
            "fused_us": stats(fused_us), "plain_us": stats(plain_us),
            "fused_e2e_us": stats(e2e_us),
            "fused_e2e_python_us": stats(py["fused"]), "plain_e2e_python_us": stats(py["plain"]),
            "fused_fits_per_s": fits / (statistics.mean(fused_us) / 1e6),
            "fused_events_per_s": n_ev / (statistics.mean(fused_us) / 1e6),
            "fused_e2e_events_per_s": n_ev / (statistics.mean(e2e_us) / 1e6),
            "plain_fits_per_s": fits / (statistics.mean(plain_us) / 1e6)})
        del pp, fp, sr
    return {"workload": label,
            "timing": "CUDA events; 256 MB written before every run (L2 cold); "
                      f"{reps} runs per size after {warmup} warm-up",
            "e2e": "fused_e2e: svt_run_host (one C call: H2D, fused path, D2H on one stream); "
                   "*_e2e_python: the same copies as torch copies around the path's calls "
                   "from Python (one svt_run, or the five per-stage calls)",
            "rows": rows}


def uneven_full(dev, flush, timer, steps=5, warmup=2):
    """The uneven workload at its full size: 65536 events per launch (16
    copies of a 4096-event draw; roads log-uniform in 1..2048, 1-16 hits per
    layer, 4096 combinations per road at most), through the fused path
    replayed from a CUDA graph, in the schedule the autotuner picks on the
    4096-event draw (every run timed after an L2 flush), the L2 flushed
    between steps as well."""
    import torch
    from paper_1311_0380_gb300 import api, autotune, synth
    spec = synth.SPECS["uneven"]
    consts = synth.make_constants(spec.n_sectors)
    base = synth.make_batch(spec, TILE_DRAW, consts, seed=spec.seed)
    b = synth.tile_batch(base, UNEVEN_EVENTS // TILE_DRAW)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg, dev)
    stream = torch.cuda.current_stream()
    fp0 = api.FusedPath(len(base.words), base.n_events, base.total_roads, dc, None, dev)
    w0, o0 = api.to_device_u32(base.words, dev), api.to_device_u64(base.event_off, dev)
    sched, tune_ms = autotune.tuned_schedule(fp0, w0, len(base.words), o0, base.n_events,
                                             cache=None, reps=2, flush=flush)
    del fp0, w0, o0
    n_words, n_events, R = len(b.words), b.n_events, b.total_roads
    fp = api.FusedPath(n_words, n_events, R, dc, sched, dev)
    d_words, d_off = api.to_device_u32(b.words, dev), api.to_device_u64(b.event_off, dev)
    g = api.GraphPath(fp, d_words, d_off)
    g.set_sizes(n_words, n_events)
    for _ in range(warmup):
        g.launch(stream)
    torch.cuda.synchronize()
    st, rec, counts = fp.result()
    assert st == api.N.STATUS_OK and int(counts[0]) == R
    fits = int(counts[2])
    assert fits == int(b.combinations(spec.max_comb).sum())
    blocks = rec.reshape(UNEVEN_EVENTS // TILE_DRAW, base.total_roads, 6)
    assert all(np.array_equal(blocks[k], blocks[0]) for k in range(1, len(blocks)))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i)
        ev[i][0].record(stream)
        g.launch(stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(c) for a, c in ev]
    fit_ms = []
    for i in range(2):
        flush.fill_(i)
        fp.run(d_words, n_words, d_off, n_events, timer=timer)
        fit_ms.append(timer.fit_ms())
    g.close()
    step_s = statistics.mean(ms) / 1e3
    fit_s = statistics.mean(fit_ms) / 1e3
    out = {"workload": f"uneven-{UNEVEN_EVENTS}ev", "events": n_events, "roads": R,
           "fits_per_step": fits, "steps": steps, "ms_per_step": step_s * 1e3,
           "fits_per_s": fits / step_s, "events_per_s": n_events / step_s,
           "fit_kernel_ms": fit_s * 1e3, "launch": "CUDA graph of the three-kernel sequence",
           "schedule": {f: getattr(sched, f) for f, _ in api.SvtSchedule._fields_},
           "tuned_on": f"{TILE_DRAW}-event draw, {tune_ms:.3f} ms per run",
           "l2": "flushed between steps (256 MB write)",
           "check": "status OK, evaluated combinations equal the closed form, all copies equal"}
    ipf = recorded_profile("warp_instructions_per_fit_uneven", UNEVEN_NOTE)
    if ipf is not None:
        ach = ipf * fits / fit_s / 1e9
        prof_sched = recorded_schedule(UNEVEN_NOTE)
        out.update({"warp_instructions_per_fit": ipf, "issue_ginst_s": ach,
                    "issue_frac": ach / ISSUE_PEAK_GINST, "ipf_schedule": prof_sched,
                    "ipf_schedule_matches": same_work_split(out["schedule"], prof_sched,
                                                            spec.max_comb)})
    del fp, d_words, d_off
    torch.cuda.empty_cache()
    return out


def main():
    args = parse_args()
    if args.sweep:
        run_sweep(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        dist_teardown(world)
        return
    import torch
    from paper_1311_0380_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec, consts, batch = workload(args, rank)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors,
                     int(spec.xft))
    dconst = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg, dev)
    n_words, n_events, R = len(batch.words), batch.n_events, batch.total_roads
    sched = api.schedule(args.warps, args.bps, args.rows,
                         args.chunk or (32 if args.lanes else 0),
                         pair_small=3 if args.lanes else 2 if args.quad else int(args.pair))
    fused = api.FusedPath(n_words, n_events, R, dconst, sched, dev)
    d_words = api.to_device_u32(batch.words, dev)
    d_off = api.to_device_u64(batch.event_off, dev)
    timer = api.FitTimer()
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)   # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_tune and not (args.warps or args.rows or args.bps or args.pair or args.quad
                                 or args.lanes or args.chunk):
        from paper_1311_0380_gb300 import autotune
        # timed as the steps are: L2 overwritten before every run
        sch, tms = autotune.tuned_schedule(fused, d_words, n_words, d_off, n_events, cache=None,
                                           flush=flush)
        fused.sched = sch
        tuned = {f: getattr(sch, f) for f, _ in api.SvtSchedule._fields_}
        tuned["tuning_ms_per_run"] = tms

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- fused path, inputs resident in HBM
    for _ in range(args.warmup):
        fused.run(d_words, n_words, d_off, n_events, timer=timer)
    torch.cuda.synchronize()
    status, rec, counts = fused.result()
    assert status == api.N.STATUS_OK, api.N.decode_status(status)
    fits_per_step = int(counts[2])
    passing = int(counts[3])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    step_ms, fit_ms = [], []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            flush.fill_(i)
            ev[i][0].record(stream)
            fused.run(d_words, n_words, d_off, n_events)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    # the fit kernel's own duration, in as many separate runs (its events
    # would keep it from overlapping its neighbours inside the timed steps)
    for i in range(args.steps):
        flush.fill_(i)
        fused.run(d_words, n_words, d_off, n_events, timer=timer)
        fit_ms.append(timer.fit_ms())
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, (job_fits, job_events) = reduce_over_ranks(
        world, sum(step_ms), [fits_per_step * args.steps, n_events * args.steps], dev)
    value = job_fits / (total_ms / 1e3)
    clock_summary = clocks.summary()

    # ---- roofline of the persistent fit kernel.  It is bound by instruction
    # issue: the headline fraction is its warp instructions per second (the
    # instructions per combination from the committed ncu summary x the
    # combinations of a step / the kernel's time) against 152 SMs x 4
    # schedulers x 2.07 GHz.  Beside it: what the GPU measurably sustains
    # (svt_pipe_peak: int32 3-input adds, multiply-adds, both, and the fp32
    # FMA stream that shows the schedulers' issue rate), the algorithmic
    # throughput in direct-form operations (57 per combination; the kernel
    # shares partial sums and executes far fewer, so this is not a
    # utilisation) and the HBM traffic against the measured copy bandwidth.
    pipe = {name: api.pipe_peak(mode)[0] for mode, name in
            ((0, "int32_add3"), (1, "int32_imad"), (2, "int32_add3_imad"), (3, "fp32_fma"))}
    issue_measured = pipe["fp32_fma"] / 32 / 1e9
    fit_mean_s = statistics.mean(fit_ms) / 1e3
    profiled = args.workload == "scaled" and args.events == 3000
    algorithmic_tops = fits_per_step * OPS_PER_FIT / fit_mean_s / 1e12
    traffic = recorded_traffic() if profiled else None
    ipf = recorded_profile("warp_instructions_per_fit") if profiled else None
    hbm_peak = measured_hbm_peak()
    if ipf is not None:
        ach = ipf * fits_per_step / fit_mean_s / 1e9
        prof_sched = recorded_schedule()
        run_sched = {f: getattr(fused.sched, f) for f, _ in api.SvtSchedule._fields_} \
            if fused.sched is not None else None
        roofline = {"bound": "alu", "achieved": ach, "peak": ISSUE_PEAK_GINST,
                    "unit": "G warp-instructions/s", "frac": ach / ISSUE_PEAK_GINST,
                    "peak_source": "derived: 152 SM x 4 schedulers x 2.07 GHz (issue rate)",
                    "warp_instructions_per_fit": ipf,
                    "frac_of_measured_issue": ach / issue_measured,
                    # the schedule of the ncu figure, and whether the timed
                    # schedule splits the work the same way (else the
                    # instructions per combination are those of the other)
                    "ipf_schedule": prof_sched,
                    "ipf_schedule_matches": same_work_split(run_sched, prof_sched,
                                                            spec.max_comb)}
    else:
        # no ncu figure for this kernel source and workload: the direct-form
        # algorithmic rate against the int32 unit count, labelled as such
        roofline = {"bound": "alu", "achieved": algorithmic_tops, "peak": ALU_PEAK_TOPS,
                    "unit": "Tops/s", "frac": algorithmic_tops / ALU_PEAK_TOPS,
                    "peak_source": "derived: 152 SM x 128 int32 lanes x 2.07 GHz; achieved = "
                                   "57 direct-form ops per combination, not a utilisation"}
    roofline.update({
        "traffic": traffic, "kernel": "k_fit_persistent", "fit_kernel_ms": fit_mean_s * 1e3,
        "algorithmic_tops": algorithmic_tops, "ops_per_fit": OPS_PER_FIT,
        "measured_issue_ginst_s": issue_measured,
        "measured_int32_add3_tlanes_s": pipe["int32_add3"] / 1e12,
        "measured_int32_imad_tlanes_s": pipe["int32_imad"] / 1e12,
        "measured_int32_mixed_tlanes_s": pipe["int32_add3_imad"] / 1e12,
        "measured_fp32_fma_tlanes_s": pipe["fp32_fma"] / 1e12,
        "hbm_gbs": (traffic / fit_mean_s / 1e9) if traffic else None,
        "hbm_frac": (traffic / fit_mean_s / 1e9 / hbm_peak) if traffic else None,
        "hbm_peak_gbs": hbm_peak})

    # ---- the uneven workload at its full size (65536 events per launch)
    uneven = None
    if rank == 0 and not args.no_uneven and args.workload == "scaled":
        uneven = uneven_full(dev, flush, timer)

    # ---- end to end from pinned host memory (fused, copies overlapped with compute)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, spec, consts, dconst, fused.sched, rank, world, dev, barrier)

    # ---- plain per-stage path beside it
    plain = None
    if not args.no_plain:
        pp = api.PlainPath(n_words, n_events, R, fits_per_step, dconst, dev)
        for _ in range(args.warmup):
            pp.run(d_words, n_words, d_off, n_events)
        torch.cuda.synchronize()
        pst, prec, _ = pp.result()
        assert pst == api.N.STATUS_OK and np.array_equal(prec, rec), "plain path differs"
        evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i)
            evp[i][0].record(stream)
            pp.run(d_words, n_words, d_off, n_events, fit_events=evf[i])
            evp[i][1].record(stream)
        torch.cuda.synchronize()
        pms = [a.elapsed_time(b) for a, b in evp]
        fms = statistics.mean(a.elapsed_time(b) for a, b in evf) / 1e3
        hbm_peak = measured_hbm_peak()
        achieved_gbs = fits_per_step * PLAIN_BYTES_PER_FIT / fms / 1e9
        plain = {"value": fits_per_step / (statistics.mean(pms) / 1e3), "unit": UNIT,
                 "ms_per_step": statistics.mean(pms),
                 "roofline_fit": {"bound": "hbm", "kernel": "k_fit_plain",
                                  "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": achieved_gbs / hbm_peak,
                                  "bytes_per_fit": PLAIN_BYTES_PER_FIT,
                                  "fit_kernel_ms": fms * 1e3,
                                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}}
        if not args.no_e2e:
            h_words, h_off = api.HostRunner.pin_batch(batch.words, batch.event_off)
            prun = api.HostRunner(pp, stream)
            for _ in range(args.warmup):
                prun.submit(h_words, h_off, R)
                prun.wait()
            lat = []
            for i in range(args.steps):
                flush.fill_(i)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                prun.submit(h_words, h_off, R)
                b.record(stream)
                prun.wait()
                lat.append(a.elapsed_time(b) * 1e3)
            plain["e2e_p50_us"] = percentile(lat, 50)
            plain["e2e_p99_us"] = percentile(lat, 99)
        del pp

    # ---- the scaled workload's batch sizes, fused beside plain, and those of
    # the paper's shape (events of 32 roads x 2^6 combinations, its Sec. 4.1)
    batch_sweep = paper_sweep = None
    if rank == 0 and not args.no_batch_sweep and args.workload == "scaled" and n_events >= 3000:
        batch_sweep = batch_size_sweep(spec, batch, dconst, dev, flush)
        from paper_1311_0380_gb300 import synth
        pspec = synth.SPECS["paper"]
        pconsts = synth.make_constants(pspec.n_sectors)
        pcfg = api.config(15, 15, pconsts.chi2_cut_99, pspec.max_comb, 5, pspec.n_sectors)
        pdconst = api.DeviceConstants.from_numpy(pconsts.F, pconsts.q, pcfg, dev)
        pbatch = synth.make_batch(pspec, max(PAPER_BATCH_SIZES), pconsts)
        paper_sweep = batch_size_sweep(pspec, pbatch, pdconst, dev, flush, PAPER_BATCH_SIZES,
                                       "paper shape (32 roads of 64 combinations an event), "
                                       "first N events of a 3000-event batch")

    serve_out = None
    if rank == 0 and not args.no_serve:
        serve_out = serving(dev, args.serve_short)

    calib_out = None
    if rank == 0 and not args.no_calib:
        calib_out = calibration(dev)

    cpu = cpu_omp = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(spec, consts, batch)
        cpu_omp = cpu_baseline_omp(spec, consts, batch)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"{args.workload}-{n_events}ev", "events": n_events, "roads": R,
                       "fits_per_step": fits_per_step, "roads_passing": passing,
                       "job_fits_per_step": job_fits // args.steps,
                       "sectors": spec.n_sectors, "max_comb": spec.max_comb,
                       "l2": "flushed between steps (256 MB write)",
                       "schedule": tuned if tuned else {"warps": args.warps,
                                                        "blocks_per_sm": args.bps,
                                                        "rows": args.rows}},
            "events_per_s": job_events / (total_ms / 1e3),
            "latency_us": {"p50": percentile([m * 1e3 for m in step_ms], 50),
                           "p99": percentile([m * 1e3 for m in step_ms], 99)},
            "e2e": e2e, "plain": plain, "roofline": roofline, "cpu_baseline": cpu,
            "cpu_baseline_omp": cpu_omp, "uneven": uneven, "batch_sizes": batch_sweep,
            "paper_batch_sizes": paper_sweep,
            "serving": serve_out,
            "calibration": calib_out,
            "clocks": clock_summary,
            "gpu_launches": api.FUSED_LAUNCHES_PER_RUN * args.steps,
        }
        print(json.dumps(line))
    dist_teardown(world)


if __name__ == "__main__":
    main()
