"""Track-trigger pairing of layers 4 and 5 (xft_pairs): the fused and plain
CUDA paths against the oracle, bit for bit, on paired batches with pairing on
and off, and the status key of rule V11 on corrupted and hand-written
streams."""
import numpy as np
import pytest

import oracle
from svt_testlib import assert_same, batch_for, cfg_pair, gpu_run, oracle_run
from test_oracle_pins import tokens_to_words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
@pytest.mark.parametrize("xft", [1, 0])
def test_paired_batch(path, xft):
    spec, consts, b = batch_for("xft", 200)
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb, xft_pairs=xft)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    assert key == oracle.KEY_OK
    st, got, extra = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, path,
                             comb_cap=int(b.combinations(spec.max_comb).sum()) * 8)
    assert_same(st, got, key, rec, f"xft={xft} {path}")
    if path == "fused":
        fits = int(b.combinations(spec.max_comb).sum()) if xft else \
            int(np.minimum(np.prod(np.maximum(b.n_hits, 1), axis=1), spec.max_comb).sum())
        assert int(extra[2]) == fits   # evaluated combinations


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_paired_batch_split_roads_and_caps(path):
    """Caps and split roads (small_max) under pairing."""
    from paper_1311_0380_gb300 import api
    spec, consts, b = batch_for("xft", 60)
    for max_comb in (7, 100, 262144):
        cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=max_comb, xft_pairs=1)
        key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
        st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, path,
                             sched=api.schedule(rows_per_item=4, small_max=64),
                             comb_cap=int(b.combinations(max_comb).sum()) + 1)
        assert_same(st, got, key, rec, f"cap {max_comb}")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_unpaired_road_is_reported(path):
    spec, consts, b = batch_for("xft", 40)
    w = b.words.copy()
    t = w >> 30
    layer = (w >> 27) & 7
    # turn the first layer-5 hit of some road into a layer-4 hit: the layers
    # stay sorted, but the road now has one layer-4 hit more than layer-5 hits
    pos = np.flatnonzero((t == 0) & (layer == 5))
    first5 = pos[np.concatenate([[True], np.diff(pos) > 1])]
    i = int(first5[len(first5) // 2])
    w[i] = (w[i] & ~np.uint32(7 << 27)) | np.uint32(4 << 27)
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb, xft_pairs=1)
    key, _ = oracle_run(w, b.event_off, consts.F, consts.q, ocfg)
    assert oracle.decode_key(key)[1] == oracle.E_XFT_UNPAIRED
    st, _, _ = gpu_run(w, b.event_off, consts.F, consts.q, cfg, path)
    assert st == key
    # without pairing the same words are valid
    cfg0, ocfg0 = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key0, rec0 = oracle_run(w, b.event_off, consts.F, consts.q, ocfg0)
    st0, got0, _ = gpu_run(w, b.event_off, consts.F, consts.q, cfg0, path,
                           comb_cap=int(np.prod(np.maximum(b.n_hits, 1), axis=1).sum()) * 2)
    assert_same(st0, got0, key0, rec0, "pairing off")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_hand_written_pairing_cases(path):
    ev = ["E:1:3",
          "R:0:1", "H:0:5", "H:1:5", "H:2:5", "H:3:5", "H:4:1", "H:4:2", "H:5:9", "H:5:8",
          "R:0:2", "H:0:5", "H:4:1", "H:4:2", "H:5:9",
          "R:0:3", "H:0:5", "H:1:5"]
    F = np.zeros((1, 64, 6, 6), np.int16)
    q = np.zeros((1, 64, 6), np.int16)
    cases = [(ev, 1), (["E:1:1", "R:0:1", "H:0:5", "H:5:9"], 1)]
    late = list(ev)
    late[16] = "HX:6:0:5"
    cases.append((late, 1))
    early = list(ev)
    early[2] = "HX:6:0:5"
    cases.append((early, 1))
    cases.append((ev, 0))
    cases.append((["E:1:1", "R:0:1"] + ["H:4:1"] * 17 + ["H:5:2"] * 2, 1))   # V8 wins
    # an event header inside a road's hits ends its run: the hits after it
    # belong to no road (V4), and the run before it is paired
    cases.append((["E:1:1", "R:0:1", "H:4:1", "H:5:2", "E:2:0", "H:4:3"], 1))
    cases.append((["E:1:1", "R:0:1", "H:4:1", "H:5:2", "T1", "H:5:3", "H:5:3"], 1))
    for toks, xft in cases:
        w = tokens_to_words(toks)
        starts = [i for i, t in enumerate(toks) if t.startswith("E:")]
        off = np.array(starts + [len(w)], np.uint64)
        cfg, ocfg = cfg_pair(n_sectors=1, min_layers=0, xft_pairs=xft)
        key, rec = oracle_run(w, off, F, q, ocfg)
        st, got, _ = gpu_run(w, off, F, q, cfg, path)
        assert_same(st, got, key, rec, str((toks, xft)))


def test_config_struct_and_limits():
    import ctypes
    from paper_1311_0380_gb300 import _native as N, api
    assert ctypes.sizeof(N.SvtConfig) == 7 * 4
    assert ctypes.sizeof(N.SvtSchedule) == 6 * 4
    spec, consts, b = batch_for("xft", 2)
    cfg, _ = cfg_pair(n_sectors=512, xft_pairs=2)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    fp = api.FusedPath(len(b.words), b.n_events, b.total_roads, dc)
    with pytest.raises(N.SvtError, match="BAD_CONFIG"):
        fp.run(api.to_device_u32(b.words), len(b.words), api.to_device_u64(b.event_off), b.n_events)
