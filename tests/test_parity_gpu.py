"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Every case runs the same seeded batch through libsvt.so and through the
oracle and compares the status key and every output word.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1311_0380_gb300 import synth
from svt_testlib import assert_same, batch_for, cfg_pair, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_0380_gb300 import api
    api.svt_version()   # loads libsvt.so or fails loudly


CONSTS = {}


def consts_for(S):
    if S not in CONSTS:
        CONSTS[S] = synth.make_constants(S)
    return CONSTS[S]


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_small_batch(path):
    spec, consts, b = batch_for("small", 100, consts_for(64))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb, n_sectors=64)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, path)
    assert_same(st, got, key, rec, "small/" + path)
    assert np.any(rec[:, 0] >> 24 & 1) and not np.all(rec[:, 0] >> 24 & 1)


@pytest.mark.parametrize("n_events", [1, 10, 100, 1000, 3000])
def test_scaled_batch_fused(n_events):
    spec, consts, b = batch_for("scaled", n_events, consts_for(512))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    st, got, counts = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused")
    assert_same(st, got, key, rec, f"scaled{n_events}")
    assert counts[0] == b.total_roads
    assert counts[2] == b.combinations(spec.max_comb).sum()
    assert counts[3] == int(np.sum(rec[:, 0] >> 24 & 1))


@pytest.mark.parametrize("n_events", [1, 100, 1000])
def test_scaled_batch_plain(n_events):
    spec, consts, b = batch_for("scaled", n_events, consts_for(512))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    n_comb = int(b.combinations(spec.max_comb).sum())
    st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "plain", comb_cap=n_comb)
    assert_same(st, got, key, rec, f"plain{n_events}")


def test_paper_shape_3000_events():
    # 2048 combinations per event, 3000 events: the paper's largest sample
    spec, consts, b = batch_for("paper", 3000, consts_for(512))
    assert int(b.combinations().sum()) == 2048 * 3000
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    for path in ("fused", "plain", "fused_pair", "fused_quad", "fused_lanes"):
        st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, path,
                             comb_cap=2048 * 3000)
        assert_same(st, got, key, rec, "paper/" + path)


@pytest.mark.parametrize("group", [1, 2, 3])
def test_grouped_roads_in_mixed_shapes(group):
    """Events of the paper's shape (runs of identical tiny roads), of the
    small workload (tiny roads of mixed geometry) and of the scaled workload
    (mostly larger roads) interleaved in one batch: with pairs (group 1) or
    also quads (group 2) the chunks mix quads, pairs and whole-warp roads;
    with one tiny road per lane (group 3) lanes of different geometry run
    side by side and the chunk's other roads follow one per warp.  Every
    record equals the oracle's."""
    from paper_1311_0380_gb300 import api
    consts = consts_for(512)
    parts = [synth.make_batch(name, n, consts, seed=70 + i)
             for i, (name, n) in enumerate((("paper", 40), ("small", 60), ("scaled", 30)))]
    events = []
    for bt in parts:
        for e in range(bt.n_events):
            events.append(bt.words[int(bt.event_off[e]):int(bt.event_off[e + 1])])
    order = np.random.default_rng(5).permutation(len(events))
    words = np.concatenate([events[i] for i in order]).astype(np.uint32)
    off = np.zeros(len(events) + 1, np.uint64)
    off[1:] = np.cumsum([len(events[i]) for i in order])
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=262144)
    key, rec = oracle_run(words, off, consts.F, consts.q, ocfg)
    for chunk in ((4, 13, 32) if group == 3 else (4, 8, 13)):
        st, got, _ = gpu_run(words, off, consts.F, consts.q, cfg, "fused",
                             sched=api.schedule(8, 0, 16, chunk, 4096, group))
        assert_same(st, got, key, rec, f"group{group}/chunk{chunk}")


def test_uneven_batch_capped():
    spec, consts, b = batch_for("uneven", 48, consts_for(512))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused")
    assert_same(st, got, key, rec, "uneven")
    assert np.mean(((rec[:, 0] >> 24) & oracle.F_OVERFLOW) > 0) > 0.5


@pytest.mark.parametrize("sched", [(1, 1, 1, 1, 1), (4, 3, 7, 3, 100), (16, 1, 64, 32, 64),
                                   (8, 4, 32, 8, 1 << 30), (2, 8, 2, 2, 33), (8, 0, 16, 4, 4096),
                                   (8, 0, 16, 4, 4096, 1), (4, 3, 7, 3, 100, 1),
                                   (16, 1, 64, 32, 64, 1), (2, 8, 2, 2, 33, 1), (1, 1, 1, 2, 1, 1),
                                   (8, 0, 16, 8, 4096, 2), (4, 3, 7, 5, 100, 2),
                                   (1, 1, 1, 4, 1, 2), (8, 0, 16, 32, 4096, 3),
                                   (4, 3, 7, 13, 100, 3), (1, 1, 1, 32, 1, 3),
                                   (12, 1, 64, 1, 64, 3), (8, 0, 256, 4, 1024),
                                   (4, 3, 1000, 3, 100), (2, 1, 129, 2, 64, 1)])
def test_schedules_give_identical_results(sched):
    from paper_1311_0380_gb300 import api
    spec, consts, b = batch_for("scaled", 60, consts_for(512))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    st, got, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused",
                         sched=api.schedule(*sched))
    assert_same(st, got, key, rec, f"sched{sched}")


@pytest.mark.parametrize("sched", [(1, 1, 16, 4, 4096), (1, 1, 16, 4, 4096, 1), (1, 1, 8, 1, 64),
                                   (1, 1, 4, 3, 300, 1), (1, 1, 16, 8, 4096, 2),
                                   (1, 1, 4, 5, 300, 2), (1, 1, 16, 32, 4096, 3),
                                   (1, 1, 4, 7, 300, 3)])
def test_record_lists_fill_and_flush(sched):
    """One warp per SM, so that every warp finishes well over 32 roads: its
    list of finished roads fills and is written out many times in the middle
    of its work (also with two paired roads arriving at a nearly full list,
    and with split roads retired into a full list)."""
    from paper_1311_0380_gb300 import api
    spec, consts, b = batch_for("scaled", 300, consts_for(512))
    assert b.total_roads > 152 * 64
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    st, got, counts = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused",
                              sched=api.schedule(*sched))
    assert_same(st, got, key, rec, f"sched{sched}")
    assert int(counts[3]) == int(np.sum(((rec[:, 0] >> 24) & oracle.F_PASS) > 0))


def test_schedule_limits_are_checked():
    from paper_1311_0380_gb300 import api
    spec, consts, b = batch_for("scaled", 4, consts_for(512))
    cfg, _ = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    for bad in (api.schedule(pair_small=4), api.schedule(warps_per_block=17),
                api.schedule(warps_per_block=13, pair_small=3),
                api.schedule(roads_per_chunk=33), api.schedule(rows_per_item=1025)):
        with pytest.raises(RuntimeError, match="BAD_ARG"):
            gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused", sched=bad)
    # one road per lane reads the constants as 32-bit pairs: constants that
    # start 2 bytes past an alignment boundary are refused before any launch
    import torch
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    F2 = torch.empty(dc.F.numel() + 2, dtype=torch.int16, device=dc.F.device)
    F2[1:1 + dc.F.numel()].copy_(dc.F.reshape(-1))
    q2 = torch.empty(dc.q.numel() + 2, dtype=torch.int16, device=dc.q.device)
    q2[1:1 + dc.q.numel()].copy_(dc.q.reshape(-1))
    R = api.roads_in(b.words, b.event_off)
    fp = api.FusedPath(len(b.words), b.n_events, R, dc)
    dw, de = api.to_device_u32(b.words), api.to_device_u64(b.event_off)
    for Fp, qp in ((F2[1:], dc.q), (dc.F, q2[1:])):
        with pytest.raises(RuntimeError, match="BAD_ARG"):
            api.svt_run(dw, len(b.words), de, b.n_events, Fp, qp, cfg, R, fp.out, fp.event_road,
                        fp.counts, fp.status, fp.workspace, sched=api.schedule(pair_small=3))
    # ... and the same buffers aligned run
    api.svt_run(dw, len(b.words), de, b.n_events, dc.F, dc.q, cfg, R, fp.out, fp.event_road,
                fp.counts, fp.status, fp.workspace, sched=api.schedule(pair_small=3))
    torch.cuda.synchronize()
    assert int(api.u64(fp.status)[0]) == api.N.STATUS_OK


# ----------------------------------------------------------------------------- edge cases
def words_of(events):
    """events: list of (event_id, [(sector, road_id, [(layer, coord), ...]), ...])"""
    words, off = [], [0]
    for eid, roads in events:
        words.append(int(synth.event_word(eid, len(roads))))
        for sec, rid, hits in roads:
            words.append(int(synth.road_word(sec, rid)))
            words.extend(int(synth.hit_word(l, c)) for l, c in sorted(hits, key=lambda h: h[0]))
        off.append(len(words))
    return np.array(words, np.uint32), np.array(off, np.uint64)


def random_consts(S, seed, scale=32768):
    rng = np.random.default_rng(seed)
    F = rng.integers(-scale, scale, (S, 64, 6, 6)).astype(np.int16)
    q = rng.integers(-scale, scale, (S, 64, 6)).astype(np.int16)
    return F, q


def test_plain_fit_tiles_over_many_and_few_roads():
    """The plain fit stages the rows of a tile of 2048 combinations when the
    tile spans at most 64 roads and reads them directly otherwise: runs of
    one-combination roads (direct), of 2048-combination roads (one road per
    tile), of 48-combination roads (about 43 per tile) and a mix, with
    missing layers and random constants, against the oracle, with
    capacities that leave a ragged last tile."""
    rng = np.random.default_rng(11)
    S = 8
    F, q = random_consts(S, 12)
    roads, rid = [], 0

    def road(n_per_layer):
        nonlocal rid
        hits = [(l, int(rng.integers(0, 32768))) for l in range(6) for _ in range(n_per_layer[l])]
        rid += 1
        return (int(rng.integers(0, S)), rid % 4096, hits)

    roads += [road([1, 1, 1, 1, 1, 1]) for _ in range(3000)]            # C = 1
    roads += [road([2, 4, 4, 4, 4, 2]) for _ in range(4)]                # C = 2048
    roads += [road([2, 3, 2, 2, 2, 1]) for _ in range(300)]              # C = 48
    roads += [road([int(v) for v in rng.integers(0, 5, 6)]) for _ in range(700)]
    events = [(e, roads[e * 50:(e + 1) * 50]) for e in range((len(roads) + 49) // 50)]
    w, off = words_of(events)
    cfg, ocfg = cfg_pair(15, 15, 3 * 12000 ** 2, 4096, 3, S)
    key, rec = oracle_run(w, off, F, q, ocfg)
    assert key == oracle.KEY_OK
    # capacities above, at and just past the combination count (a ragged
    # last tile)
    n_comb = int(sum(np.prod([max(sum(1 for h in hits if h[0] == l), 1) for l in range(6)])
                     for _, _, hits in roads))
    for cap in (len(roads) * 4096, len(roads) * 4096 + 1, n_comb + 3 - (n_comb + 3) % 4,
                n_comb):
        st, got, _ = gpu_run(w, off, F, q, cfg, "plain", comb_cap=cap)
        assert_same(st, got, key, rec, f"plain tiles, capacity {cap}")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_empty_batch_and_events_without_roads(path):
    F, q = random_consts(4, 1)
    cfg, ocfg = cfg_pair(n_sectors=4)
    w = np.zeros(0, np.uint32)
    off = np.zeros(1, np.uint64)
    st, got, _ = gpu_run(w, off, F, q, cfg, path)
    assert st == oracle.KEY_OK
    w, off = words_of([(1, []), (2, []), (3, [])])
    key, rec = oracle_run(w, off, F, q, ocfg)
    st, got, _ = gpu_run(w, off, F, q, cfg, path)
    assert_same(st, got, key, rec, "no roads")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_missing_layers_patterns_and_no_hits(path):
    rng = np.random.default_rng(3)
    F, q = random_consts(8, 2, scale=3000)
    roads = []
    for rid in range(300):
        n = rng.integers(0, 4, 6)
        if rid % 50 == 0:
            n[:] = 0
        hits = [(l, int(rng.integers(0, 32768))) for l in range(6) for _ in range(n[l])]
        roads.append((int(rng.integers(0, 8)), rid, hits))
    events = [(e, roads[e * 30:(e + 1) * 30]) for e in range(10)]
    w, off = words_of(events)
    for min_layers in (0, 3, 5, 6):
        cfg, ocfg = cfg_pair(chi2_cut=200000000, max_comb=50, min_layers=min_layers, n_sectors=8)
        key, rec = oracle_run(w, off, F, q, ocfg)
        st, got, _ = gpu_run(w, off, F, q, cfg, path, comb_cap=300 * 64)
        assert_same(st, got, key, rec, f"min_layers{min_layers}")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_ties_and_extreme_constants(path):
    rng = np.random.default_rng(4)
    S = 2
    F, q = random_consts(S, 5)
    F[:, :, 3:, :] = rng.integers(-2, 3, (S, 64, 3, 6))      # tiny chi rows: many equal chi2
    roads = []
    for rid in range(400):
        n = rng.integers(1, 5, 6)
        base = int(rng.integers(0, 32768))
        hits = [(l, base if rng.random() < 0.6 else int(rng.integers(0, 32768)))
                for l in range(6) for _ in range(n[l])]
        roads.append((int(rng.integers(0, S)), rid, hits))
    w, off = words_of([(e, roads[e * 40:(e + 1) * 40]) for e in range(10)])
    for cut in (0, 5, 1000, 0xFFFFFFFF):
        for oshift, qshift in ((15, 15), (9, 0), (9, 24), (31, 24), (12, 20)):
            cfg, ocfg = cfg_pair(oshift, qshift, cut, 300, 5, S)
            key, rec = oracle_run(w, off, F, q, ocfg)
            st, got, _ = gpu_run(w, off, F, q, cfg, path, comb_cap=400 * 300)
            assert_same(st, got, key, rec, f"cut{cut} os{oshift} qs{qshift}")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_chi_components_at_the_clamp_boundary(path):
    """chi components straddling +-32767 / +-32768 (the clamp of Eq. 2's
    chi-square), with cuts just below, at and above 32767^2: the range test of
    the small-cut kernels and the clamped sum of the large-cut kernels both
    agree with the oracle's clamped reading, ties included."""
    rng = np.random.default_rng(11)
    S = 2
    F = np.zeros((S, 64, 6, 6), np.int16)
    q = np.zeros((S, 64, 6), np.int16)
    F[:, :, :3, :] = rng.integers(-2000, 2000, (S, 64, 3, 6))
    # oshift = qshift = 15: y_k = q_k + floor(sum_l F_kl x_l / 2^15), x_l < 2^15
    F[0, :, 3, :] = rng.integers(0, 3, (64, 6))      # y_3 in [32764, 32776)
    q[0, :, 3] = 32764
    F[1, :, 3, :] = -rng.integers(0, 3, (64, 6))     # y_3 in (-32776, -32764]
    q[1, :, 3] = -32764
    F[:, :, 4:, :] = rng.integers(-1, 2, (S, 64, 2, 6))   # y_4, y_5 in [-6, 6)
    roads = []
    for rid in range(600):
        n = rng.integers(1, 4, 6)
        hits = [(l, int(rng.integers(0, 32768))) for l in range(6) for _ in range(n[l])]
        roads.append((rid % S, rid, hits))
    w, off = words_of([(e, roads[e * 50:(e + 1) * 50]) for e in range(12)])
    c = 32767 * 32767
    n_pass = []
    for cut in (c - 70000, c - 1, c, c + 100, 0xFFFFFFFF):
        cfg, ocfg = cfg_pair(15, 15, cut, 729, 6, S)
        key, rec = oracle_run(w, off, F, q, ocfg)
        n_pass.append(int(np.count_nonzero(rec[:, 0] & (1 << 24))))
        st, got, _ = gpu_run(w, off, F, q, cfg, path, comb_cap=600 * 729)
        assert_same(st, got, key, rec, f"cut {cut}")
    assert 0 < n_pass[0] < n_pass[1] < n_pass[2] < n_pass[3]   # each cut decides roads


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_maximum_hits_per_layer(path):
    # 16 hits in every layer: 16^6 combinations, capped
    rng = np.random.default_rng(6)
    F, q = random_consts(1, 7, scale=20000)
    roads = [(0, rid, [(l, int(rng.integers(0, 32768))) for l in range(6) for _ in range(16)])
             for rid in range(6)]
    w, off = words_of([(0, roads)])
    for cap in (1, 31, 33, 4096, 70000):
        cfg, ocfg = cfg_pair(max_comb=cap, n_sectors=1, chi2_cut=0xFFFFFFFF)
        key, rec = oracle_run(w, off, F, q, ocfg)
        st, got, _ = gpu_run(w, off, F, q, cfg, path, comb_cap=6 * cap)
        assert_same(st, got, key, rec, f"cap{cap}")
        assert np.all(rec[:, 0] >> 24 & oracle.F_OVERFLOW)


def test_uneven_batch_split_and_whole_agree():
    from paper_1311_0380_gb300 import api
    spec, consts, b = batch_for("uneven", 12, consts_for(512))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    for small_max in (1, 500, 4096):
        st, got, counts = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused",
                                  sched=api.schedule(rows_per_item=8, small_max=small_max))
        assert_same(st, got, key, rec, f"small_max{small_max}")
        assert (counts[1] > 0) == (small_max < 4096)


def test_uncapped_giant_road_fused():
    # one road of 16^5 * 8 = 8.4M combinations next to small ones
    rng = np.random.default_rng(8)
    F, q = random_consts(1, 9, scale=20000)
    big = (0, 1, [(l, int(rng.integers(0, 32768))) for l in range(6) for _ in range(16 if l else 8)])
    small = [(0, 2 + i, [(l, int(rng.integers(0, 32768))) for l in range(6)]) for i in range(5)]
    w, off = words_of([(0, small[:2] + [big] + small[2:])])
    cfg, ocfg = cfg_pair(max_comb=1 << 24, n_sectors=1, chi2_cut=0xFFFFFFFF)
    key, rec = oracle_run(w, off, F, q, ocfg)
    st, got, _ = gpu_run(w, off, F, q, cfg, "fused")
    assert_same(st, got, key, rec, "giant")


@pytest.mark.parametrize("path", ["fused", "plain", "fused_pair", "fused_quad", "fused_lanes"])
def test_validation_cases_match_oracle(path):
    from test_oracle_pins import tokens_to_words
    data = json.load(open(os.path.join(GOLDEN, "validation_cases.json")))
    F, q = random_consts(64, 10)
    for case in data["cases"]:
        w = tokens_to_words(case["words"])
        off = np.array(case["offsets"], np.uint64)
        xft = case.get("xft_pairs", 0)
        cfg, ocfg = cfg_pair(n_sectors=case["n_sectors"], min_layers=0, xft_pairs=xft)
        key = oracle.validate(w, off, case["n_sectors"], xft_pairs=xft)
        if key == oracle.KEY_OK:
            key, rec = oracle_run(w, off, F, q, ocfg)
        else:
            rec = None
        st, got, _ = gpu_run(w, off, F, q, cfg, path, road_cap=len(w) + 1)
        assert_same(st, got, key, rec, case["name"])


def test_random_corruptions_match_oracle():
    rng = np.random.default_rng(11)
    spec, consts, b = batch_for("small", 30, consts_for(64))
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb, n_sectors=64)
    for trial in range(40):
        w = b.words.copy()
        for _ in range(int(rng.integers(1, 4))):
            i = int(rng.integers(0, len(w)))
            w[i] ^= np.uint32(1) << np.uint32(int(rng.integers(0, 32)))
        key = oracle.validate(w, b.event_off, 64)
        rec = oracle_run(w, b.event_off, consts.F, consts.q, ocfg)[1] if key == oracle.KEY_OK else None
        st, got, _ = gpu_run(w, b.event_off, consts.F, consts.q, cfg, "fused", road_cap=len(w))
        assert_same(st, got, key, rec, f"corrupt{trial}")


def test_road_capacity_overflow_is_reported():
    spec, consts, b = batch_for("small", 5, consts_for(64))
    cfg, _ = cfg_pair(n_sectors=64)
    st, _, _ = gpu_run(b.words, b.event_off, consts.F, consts.q, cfg, "fused", road_cap=7)
    assert st & 0xFF == 9



def test_uneven_full_size_65536_events():
    """The uneven workload at its full size, 65536 events per launch (16 copies
    of a 4096-event draw: 17 million roads, 69 billion evaluated
    combinations), through the fused path in the schedule the bench uses:
    the first copy's records equal the oracle's records of the whole
    4096-event draw (one event per host thread, 4.4 billion fits), and every
    other copy's records equal the first copy's, so every one of the 17
    million records is checked."""
    import torch
    from paper_1311_0380_gb300 import api
    spec = synth.SPECS["uneven"]
    consts = consts_for(512)
    base = synth.make_batch(spec, 4096, consts)
    b = synth.tile_batch(base, 16)
    R0 = base.total_roads
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    fp = api.FusedPath(len(b.words), b.n_events, b.total_roads, dc)
    fp.run(api.to_device_u32(b.words), len(b.words), api.to_device_u64(b.event_off), b.n_events)
    torch.cuda.synchronize()
    st, rec, counts = fp.result()
    assert st == oracle.KEY_OK
    assert counts[0] == b.total_roads == 16 * R0
    assert counts[2] == int(b.combinations(spec.max_comb).sum())
    blocks = rec.reshape(16, R0, 6)
    assert all(np.array_equal(blocks[k], blocks[0]) for k in range(1, 16))
    key, want = oracle.run(base.words, base.event_off, consts.F, consts.q, ocfg, omp=True)
    assert key == oracle.KEY_OK
    assert_same(st, blocks[0], key, want, "uneven 4096-event draw")
    assert np.mean(((want[:, 0] >> 24) & oracle.F_OVERFLOW) > 0) > 0.5   # mostly capped roads
