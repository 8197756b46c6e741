"""Shared helpers of the GPU parity tests: run a batch through the CUDA path
(fused or plain) and through the oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_1311_0380_gb300 import synth


def cfg_pair(oshift=15, qshift=15, chi2_cut=0xFFFFFFFF, max_comb=262144, min_layers=5,
             n_sectors=512, xft_pairs=0):
    from paper_1311_0380_gb300 import api
    return (api.config(oshift, qshift, chi2_cut, max_comb, min_layers, n_sectors, xft_pairs),
            oracle.config(oshift, qshift, chi2_cut, max_comb, min_layers, n_sectors, xft_pairs))


def oracle_run(words, event_off, F, q, ocfg):
    return oracle.run(words, event_off, F, q, ocfg, omp=True)


def gpu_run(words, event_off, F, q, cfg, path="fused", sched=None, road_cap=None, comb_cap=None):
    import torch
    from paper_1311_0380_gb300 import api
    words = np.ascontiguousarray(words, np.uint32)
    event_off = np.ascontiguousarray(event_off, np.uint64)
    n_words, n_events = len(words), len(event_off) - 1
    if road_cap is None:
        road_cap = max(api.roads_in(words, event_off), 1)
    consts = api.DeviceConstants.from_numpy(F, q, cfg)
    if path in ("fused_pair", "fused_quad", "fused_lanes"):
        # the fused path with pairing of small roads (chunks of 8 roads unless
        # the test gives its own schedule); fused_quad also groups four tiny
        # roads per warp; fused_lanes fits every tiny road on a lane of its
        # own (chunks of 32 roads)
        s = sched if sched is not None else api.schedule()
        lanes = path == "fused_lanes"
        sched = api.schedule(s.warps_per_block, s.blocks_per_sm, s.rows_per_item,
                             s.roads_per_chunk or (32 if lanes else 8), s.small_max,
                             3 if lanes else 2 if path == "fused_quad" else 1)
        path = "fused"
    dw = api.to_device_u32(words if n_words else np.zeros(4, np.uint32))
    de = api.to_device_u64(event_off)
    if path == "fused":
        fp = api.FusedPath(max(n_words, 1), max(n_events, 1), road_cap, consts, sched)
        fp.run(dw, n_words, de, n_events)
        torch.cuda.synchronize()
        status, rec, counts = fp.result()
        return status, rec, counts
    if comb_cap is None:
        comb_cap = 1 << 20
    pp = api.PlainPath(max(n_words, 1), max(n_events, 1), road_cap, comb_cap, consts)
    pp.run(dw, n_words, de, n_events)
    torch.cuda.synchronize()
    status, rec, R = pp.result()
    return status, rec, pp


def assert_same(status_g, rec_g, key_o, rec_o, what=""):
    assert status_g == key_o, (what, oracle.decode_key(status_g), oracle.decode_key(key_o))
    if key_o == oracle.KEY_OK:
        assert rec_g.shape == rec_o.shape, (what, rec_g.shape, rec_o.shape)
        bad = np.flatnonzero(np.any(rec_g != rec_o, axis=1))
        assert len(bad) == 0, (what, len(bad), bad[:5], rec_g[bad[:3]], rec_o[bad[:3]])


def batch_for(name, n_events, consts=None):
    spec = synth.SPECS[name]
    if consts is None:
        consts = synth.make_constants(spec.n_sectors)
    return spec, consts, synth.make_batch(spec, n_events, consts)
