"""Batching row: one captured CUDA graph of the fused path replayed for
batches of different sizes (sizes read on the device), and the schedule
autotuner, both bit-exact with the oracle."""
import ctypes
import json

import numpy as np
import pytest

import oracle
from paper_1311_0380_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_graph_replayed_for_batches_of_different_sizes():
    import torch
    from paper_1311_0380_gb300 import api, _native as N
    consts = synth.make_constants(512)
    cfg = api.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    max_words, max_events, road_cap = 1 << 21, 512, 1 << 16
    d_words = torch.zeros(max_words, dtype=torch.int32, device="cuda")
    d_off = torch.zeros(max_events + 1, dtype=torch.int64, device="cuda")
    d_sizes = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = torch.zeros(road_cap * 6, dtype=torch.int32, device="cuda")
    ev = torch.zeros(max_events + 1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(4, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(api.svt_run_workspace_size(max_words, max_events, road_cap), dtype=torch.uint8,
                     device="cuda")
    L = N.load()
    g = ctypes.c_void_p()
    N.check(L.svt_graph_create(api._p(d_words), max_words, api._p(d_off), max_events,
                               api._p(d_sizes), api._p(dc.F), api._p(dc.q), ctypes.byref(cfg),
                               road_cap, api._p(out), api._p(ev), api._p(counts), api._p(status),
                               api._p(ws), ws.numel(), None, ctypes.byref(g)), "svt_graph_create")
    batches = [synth.make_batch("scaled", 7, consts, seed=1), synth.make_batch("uneven", 3, consts, seed=2),
               synth.make_batch("scaled", 150, consts, seed=3), synth.make_batch("small", 1, None, seed=4)]
    batches[3] = synth.make_batch(synth.BatchSpec("s512", 512, ("const", 16), ("uniform", 1, 2), 64, 9), 40, consts)
    for b in batches:
        key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q, ocfg, omp=True)
        d_words[: len(b.words)].copy_(torch.from_numpy(b.words.view(np.int32)))
        d_off[: b.n_events + 1].copy_(torch.from_numpy(b.event_off.view(np.int64)))
        d_sizes.copy_(torch.tensor([len(b.words), b.n_events], dtype=torch.int64))
        N.check(L.svt_graph_launch(g, api._stream(None)), "svt_graph_launch")
        torch.cuda.synchronize()
        assert int(api.u64(status)[0]) == key == oracle.KEY_OK
        got = api.u32(out[: b.total_roads * 6]).reshape(-1, 6)
        assert np.array_equal(got, rec)
        assert int(api.u64(counts)[0]) == b.total_roads
    # sizes above the captured capacities are refused on the device, not run
    d_sizes.copy_(torch.tensor([max_words + 1, 1], dtype=torch.int64))
    N.check(L.svt_graph_launch(g, api._stream(None)), "svt_graph_launch")
    torch.cuda.synchronize()
    assert int(api.u64(status)[0]) & 0xFF == 1
    N.check(L.svt_graph_destroy(g), "svt_graph_destroy")


def test_autotuner_picks_a_schedule_that_stays_bit_exact(tmp_path):
    import torch
    from paper_1311_0380_gb300 import api, autotune
    consts = synth.make_constants(512)
    spec = synth.SPECS["scaled"]
    b = synth.make_batch(spec, 120, consts)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q,
                          oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512), omp=True)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    fp = api.FusedPath(len(b.words), b.n_events, b.total_roads, dc)
    dw, de = api.to_device_u32(b.words), api.to_device_u64(b.event_off)
    cache = str(tmp_path / "sched.json")
    sch, ms = autotune.tuned_schedule(fp, dw, len(b.words), de, b.n_events, cache=cache, reps=1)
    assert ms > 0 and sch.warps_per_block in (4, 8, 16) and sch.rows_per_item in (8, 16, 32, 64)
    # the tuner's last run leaves a valid result (it passes no counts buffer)
    st = int(api.u64(fp.status)[0])
    got = api.u32(fp.out[: b.total_roads * 6]).reshape(-1, 6)
    assert st == key and np.array_equal(got, rec)
    fp.sched = sch
    fp.run(dw, len(b.words), de, b.n_events)
    torch.cuda.synchronize()
    st, got, _ = fp.result()
    assert st == key and np.array_equal(got, rec)
    sch2, ms2 = autotune.tuned_schedule(fp, dw, len(b.words), de, b.n_events, cache=cache)
    assert (sch2.warps_per_block, sch2.rows_per_item, sch2.roads_per_chunk, sch2.small_max) == \
        (sch.warps_per_block, sch.rows_per_item, sch.roads_per_chunk, sch.small_max)


def test_autotune_with_l2_flush(tmp_path):
    """Timing every run after a flush write still leaves a valid result, keys
    the cache apart from back-to-back tuning, and a flush size without a
    buffer is refused."""
    import torch
    from paper_1311_0380_gb300 import api, autotune, synth
    consts = synth.make_constants(512)
    spec = synth.SPECS["scaled"]
    b = synth.make_batch(spec, 40, consts)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q,
                          oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512), omp=True)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    fp = api.FusedPath(len(b.words), b.n_events, b.total_roads, dc)
    dw, de = api.to_device_u32(b.words), api.to_device_u64(b.event_off)
    flush = torch.empty(2 << 20, dtype=torch.int32, device="cuda")
    cache = str(tmp_path / "sched.json")
    sch, ms = autotune.tuned_schedule(fp, dw, len(b.words), de, b.n_events, cache=cache, reps=1,
                                      flush=flush)
    assert ms > 0 and sch.warps_per_block in (4, 8, 16)
    st = int(api.u64(fp.status)[0])
    got = api.u32(fp.out[: b.total_roads * 6]).reshape(-1, 6)
    assert st == key and np.array_equal(got, rec)
    table = json.load(open(cache))
    assert len(table) == 1 and next(iter(table)).endswith("|l1")
    best, bms = api.SvtSchedule(), ctypes.c_float()
    c = fp.consts
    rc = api.N.load().svt_autotune(api._p(dw), len(b.words), api._p(de), b.n_events, api._p(c.F),
                                   api._p(c.q), ctypes.byref(c.cfg), fp.road_cap, api._p(fp.out),
                                   api._p(fp.status), api._p(fp.workspace),
                                   fp.workspace.numel(), 1, None, 1 << 20, ctypes.byref(best),
                                   ctypes.byref(bms), api._stream(None))
    assert api.N.ERRORS[rc] == "BAD_ARG"


def test_streaming_runner_overlapped_steps_are_exact():
    """Batches go through svt_run_host (copy in, fused path, copy out in one
    library call) on two alternating streams, so copies and compute of
    consecutive steps overlap; the records of each step still equal the
    oracle's for that step's batch."""
    import torch
    from paper_1311_0380_gb300 import api
    consts = synth.make_constants(512)
    spec = synth.SPECS["scaled"]
    batches = [synth.make_batch(spec, 40, consts, seed=500 + k) for k in range(3)]
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    want = [oracle.run(b.words, b.event_off, consts.F, consts.q, ocfg, omp=True)[1] for b in batches]
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    runner = api.StreamingRunner(max(len(b.words) for b in batches), 40,
                                 max(b.total_roads for b in batches), dc, depth=2)
    pinned = [api.HostRunner.pin_batch(b.words, b.event_off) for b in batches]
    order = [0, 1, 2, 1, 0]
    for k in order:
        runner.submit(pinned[k][0], pinned[k][1], batches[k].total_roads)
    st, rec = runner.wait()
    assert st == oracle.KEY_OK and np.array_equal(rec, want[order[-1]])
    # the other set holds the step before
    st_prev, prev = runner.result((runner.i - 2) % runner.depth)
    assert st_prev == oracle.KEY_OK and np.array_equal(prev, want[order[-2]])


def test_run_host_single_call_matches_oracle_and_reports_bad_data():
    """svt_run_host on one stream: the records equal the oracle's; a corrupt
    batch returns the oracle's status key; a workspace sized for a smaller
    batch is refused."""
    import torch
    from paper_1311_0380_gb300 import api
    consts = synth.make_constants(512)
    spec = synth.SPECS["uneven"]
    b = synth.make_batch(spec, 5, consts, seed=77)
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, 512)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    hw, ho = api.HostRunner.pin_batch(b.words, b.event_off)
    R = b.total_roads
    ws = torch.empty(api.svt_run_host_workspace_size(len(b.words), b.n_events, R), dtype=torch.uint8,
                     device="cuda")
    h_out = torch.empty(R * 6, dtype=torch.int32, pin_memory=True)
    h_st = torch.empty(1, dtype=torch.int64, pin_memory=True)
    n = api.svt_run_host(hw, len(b.words), ho, b.n_events, dc.F, dc.q, cfg, R, h_out, h_st, ws)
    torch.cuda.synchronize()
    key, want = oracle.run(b.words, b.event_off, consts.F, consts.q, ocfg, omp=True)
    assert n == R and int(h_st.numpy().view(np.uint64)[0]) == key == oracle.KEY_OK
    assert np.array_equal(h_out.numpy().view(np.uint32).reshape(-1, 6), want)
    w2 = b.words.copy()
    w2[int(b.event_off[2]) + 1] = np.uint32(1 << 30)          # a type-1 word
    hw2, _ = api.HostRunner.pin_batch(w2, b.event_off)
    api.svt_run_host(hw2, len(w2), ho, b.n_events, dc.F, dc.q, cfg, R, h_out, h_st, ws)
    torch.cuda.synchronize()
    assert int(h_st.numpy().view(np.uint64)[0]) == oracle.validate(w2, b.event_off, 512)
    with pytest.raises(api.N.SvtError, match="BAD_ARG"):
        api.svt_run_host(hw, len(b.words), ho, b.n_events, dc.F, dc.q, cfg, R, h_out, h_st,
                         ws[: ws.numel() // 2])
