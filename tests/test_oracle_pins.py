"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against what the method and the mathematics fix:
Python big-integer evaluation of the fit formula (floor division), brute-force
enumeration of the combinations with itertools, exhaustive argmin with
injected ties, hand-worked roads (tests/golden/worked_examples.json), the
hand-written validation cases (tests/golden/validation_cases.json) and the
closed-form fit-back of noise-free linear tracks.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1311_0380_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers
def bigint_fit(F36, q6, x6, oshift, qshift):
    """The fit written with Python integers: y_k = (q_k 2^qs + sum F x) // 2^os."""
    y = []
    for k in range(6):
        acc = int(q6[k]) * (1 << qshift) + sum(int(F36[k * 6 + l]) * int(x6[l]) for l in range(6))
        y.append(acc // (1 << oshift))
    chi2 = sum(max(-32767, min(32767, v)) ** 2 for v in y[3:])
    return y, chi2


def tokens_to_words(tokens):
    out = []
    for t in tokens:
        p = t.split(":")
        if p[0] == "E":
            out.append(int(synth.event_word(int(p[1]), int(p[2]))))
        elif p[0] == "R":
            out.append(int(synth.road_word(int(p[1]), int(p[2]))))
        elif p[0] == "H":
            out.append(int(synth.hit_word(int(p[1]), int(p[2]))))
        elif p[0] == "HX":
            out.append((int(p[1]) << 27) | (int(p[2]) << 15) | int(p[3]))
        elif p[0] == "T1":
            out.append(1 << 30)
        else:
            raise ValueError(t)
    return np.array(out, np.uint32)


def table_with(sector, mask, F6x6, q6, n_sectors=1):
    F = np.zeros((n_sectors, 64, 6, 6), np.int16)
    q = np.zeros((n_sectors, 64, 6), np.int16)
    F[sector, mask] = F6x6
    q[sector, mask] = q6
    return F, q


# --------------------------------------------------------------------------- fit arithmetic
@pytest.mark.parametrize("oshift,qshift", [(15, 15), (9, 0), (31, 24), (20, 3), (12, 20)])
def test_fit_one_matches_bigint(oshift, qshift):
    rng = np.random.default_rng(11 + oshift * 100 + qshift)
    extremes_F = np.array([-32768, 32767, -1, 0, 1], np.int64)
    extremes_x = np.array([0, 32767, 1, 16384], np.int64)
    for trial in range(600):
        if trial % 3 == 0:
            F = rng.choice(extremes_F, 36)
            x = rng.choice(extremes_x, 6)
            q = rng.choice(extremes_F, 6)
        else:
            F = rng.integers(-32768, 32768, 36)
            x = rng.integers(0, 32768, 6)
            q = rng.integers(-32768, 32768, 6)
        y, chi2 = oracle.fit_one(F, q, x, oshift, qshift)
        y_ref, chi2_ref = bigint_fit(F, q, x, oshift, qshift)
        assert list(y) == y_ref
        assert chi2 == chi2_ref


def test_fit_zero_matrix_and_halving_rows():
    # F = 0: y = floor(q 2^qs / 2^os); F = 16384 on the diagonal with os = 15: y = floor(x/2)
    q = np.array([-3, 5, -32768, 32767, 0, 1], np.int16)
    y, _ = oracle.fit_one(np.zeros(36, np.int16), q, np.full(6, 32767), 15, 10)
    assert list(y) == [v * 1024 // 32768 for v in q.tolist()]
    F = np.diag([16384] * 6).astype(np.int16)
    x = np.array([0, 1, 2, 3, 32767, 32766])
    y, chi2 = oracle.fit_one(F, np.zeros(6), x, 15, 15)
    assert list(y) == [0, 0, 1, 1, 16383, 16383]
    assert chi2 == 1 + 16383 ** 2 * 2


def test_chi_clamp_at_32767():
    F = np.zeros((6, 6), np.int16)
    F[3, 0] = 32767      # y3 = floor(32767*32767/2^9) far above 32767
    F[4, 0] = -32768     # y4 far below -32767
    y, chi2 = oracle.fit_one(F, np.zeros(6), [32767, 0, 0, 0, 0, 0], 9, 0)
    assert y[3] > 32767 and y[4] < -32767
    assert chi2 == 2 * 32767 ** 2


# --------------------------------------------------------------------------- hand-worked roads
def test_worked_examples():
    data = json.load(open(os.path.join(GOLDEN, "worked_examples.json")))
    F, q = table_with(0, 63, data["constants"]["F"], data["constants"]["q"])
    for road in data["roads"]:
        cfg = oracle.config(15, 15, road["cut"], 262144, 5, 1)
        n = [len(h) for h in road["hits"]]
        rec = oracle.road(n, road["hits"], 0, road["road_id"], F, q, cfg)
        assert rec.tolist() == road["record"], road["name"]


# --------------------------------------------------------------------------- combinations
def random_road(rng, max_hits=3, allow_empty=True):
    lo = 0 if allow_empty else 1
    n = rng.integers(lo, max_hits + 1, 6)
    hits = [rng.integers(0, 32768, int(k)).tolist() for k in n]
    return n, hits


def test_combination_count_order_and_values_brute_force():
    rng = np.random.default_rng(5)
    S = 3
    F = rng.integers(-32768, 32768, (S, 64, 6, 6)).astype(np.int16)
    q = rng.integers(-32768, 32768, (S, 64, 6)).astype(np.int16)
    for _ in range(300):
        n, hits = random_road(rng)
        sector = int(rng.integers(0, S))
        cfg = oracle.config(15, 15, 0xFFFFFFFF, 1 << 24, 0, S)
        rec, chi2s, ys = oracle.road(n, hits, sector, 1, F, q, cfg, detail=True)
        mask = sum(1 << l for l in range(6) if n[l] > 0)
        ranges = [range(max(int(k), 1)) for k in n]
        combos = list(itertools.product(*ranges))      # layer 0 outermost, layer 5 fastest
        assert len(chi2s) == int(np.prod(np.maximum(n, 1)))
        assert len(chi2s) == len(combos)
        for c, idx in enumerate(combos):
            x = [hits[l][idx[l]] if n[l] > 0 else 0 for l in range(6)]
            y_ref, chi_ref = bigint_fit(F[sector, mask].ravel(), q[sector, mask], x, 15, 15)
            assert list(ys[c]) == y_ref
            assert chi2s[c] == chi_ref


def exhaustive_best(n, hits, F36, q6, cut, max_comb, oshift=15, qshift=15):
    ranges = [range(max(int(k), 1)) for k in n]
    best = None
    for c, idx in enumerate(itertools.product(*ranges)):
        if c >= max_comb:
            break
        x = [hits[l][idx[l]] if n[l] > 0 else 0 for l in range(6)]
        y, chi2 = bigint_fit(F36, q6, x, oshift, qshift)
        if chi2 <= cut and (best is None or (chi2, c) < (best[1], best[0])):
            best = (c, chi2, y[:3])
    return best


def test_select_exhaustive_with_ties():
    rng = np.random.default_rng(9)
    for trial in range(300):
        n, hits = random_road(rng, max_hits=4, allow_empty=False)
        # inject ties: repeat a coordinate inside a layer, or copy a layer's hits
        l = int(rng.integers(0, 6))
        if n[l] >= 2:
            hits[l][1] = hits[l][0]
        F = np.zeros((1, 64, 6, 6), np.int16)
        q = np.zeros((1, 64, 6), np.int16)
        small = rng.integers(-40, 41, (6, 6))
        F[0, 63] = small
        q[0, 63] = rng.integers(-2000, 2000, 6)
        chi2_all = oracle.road(n, hits, 0, 0, F, q, oracle.config(15, 15, 0xFFFFFFFF, 1 << 24, 0, 1),
                               detail=True)[1]
        cut = int(rng.choice([0, int(np.median(chi2_all)), int(chi2_all.min()), 0xFFFFFFFF]))
        max_comb = int(rng.choice([1, 3, len(chi2_all), 1 << 24]))
        cfg = oracle.config(15, 15, cut, max_comb, 0, 1)
        rec = oracle.road(n, hits, 0, 77, F, q, cfg)
        best = exhaustive_best(n, hits, F[0, 63].ravel(), q[0, 63], cut, max_comb)
        flags = rec[0] >> 24
        assert bool(flags & oracle.F_OVERFLOW) == (len(chi2_all) > max_comb)
        if best is None:
            assert rec.tolist()[1:] == [0xFFFFFFFF, 0, 0, 0, 0]
            assert not flags & oracle.F_PASS
        else:
            assert flags & oracle.F_PASS
            assert rec[1] == best[0] and rec[2] == best[1]
            assert [int(np.int32(np.uint32(v))) for v in rec[3:]] == best[2]


def test_pattern_flags():
    F = np.zeros((1, 64, 6, 6), np.int16)
    q = np.zeros((1, 64, 6), np.int16)
    # 4 layers hit, min_layers 5 -> BAD_PATTERN, nothing evaluated
    rec, chi2s, _ = oracle.road([1, 1, 1, 1, 0, 0], [[1], [2], [3], [4], [], []], 0, 3, F, q,
                                oracle.config(min_layers=5, n_sectors=1), detail=True)
    assert rec[0] >> 24 == oracle.F_BAD_PATTERN and len(chi2s) == 0
    # no hits at all with min_layers 0: one combination with x = 0 -> chi2 = 0 passes
    rec = oracle.road([0] * 6, [[]] * 6, 0, 4, F, q, oracle.config(min_layers=0, n_sectors=1))
    assert rec[0] >> 24 == oracle.F_NO_HITS | oracle.F_PASS and rec[1] == 0
    # no hits with min_layers 1 -> both flags
    rec = oracle.road([0] * 6, [[]] * 6, 0, 4, F, q, oracle.config(min_layers=1, n_sectors=1))
    assert rec[0] >> 24 == oracle.F_NO_HITS | oracle.F_BAD_PATTERN


def test_missing_layer_uses_its_mask_constants():
    # mask 0b011111 (layer 5 empty): the row of mask 31 must be used and x5 = 0
    F = np.zeros((1, 64, 6, 6), np.int16)
    q = np.zeros((1, 64, 6), np.int16)
    F[0, 31, 0, 0] = 16384
    q[0, 31, 1] = 9
    F[0, 63, 0, 0] = -16384
    rec = oracle.road([1, 1, 1, 1, 1, 0], [[100], [1], [1], [1], [1], []], 0, 0, F, q,
                      oracle.config(min_layers=5, n_sectors=1))
    assert [int(np.int32(np.uint32(v))) for v in rec[3:]] == [50, 9, 0]


# --------------------------------------------------------------------------- validation
def test_validation_cases():
    data = json.load(open(os.path.join(GOLDEN, "validation_cases.json")))
    for case in data["cases"]:
        words = tokens_to_words(case["words"])
        key = oracle.validate(words, np.array(case["offsets"], np.uint64), case["n_sectors"],
                              xft_pairs=case.get("xft_pairs", 0))
        got = oracle.decode_key(key)
        exp = None if case["expect"] is None else tuple(case["expect"])
        assert got == exp, case["name"]


def test_generated_batches_are_valid_and_parse_back():
    for name, ne in [("small", 50), ("scaled", 20), ("uneven", 2), ("paper", 5)]:
        spec = synth.SPECS[name]
        consts = synth.make_constants(spec.n_sectors)
        b = synth.make_batch(spec, ne, consts)
        assert oracle.validate(b.words, b.event_off, spec.n_sectors) == oracle.KEY_OK
        # independent parse of the words with numpy: hits per layer of every road
        t = b.words >> 30
        road_pos = np.flatnonzero(t == 2)
        assert len(road_pos) == b.total_roads
        layer = (b.words >> 27) & 7
        road_of_word = np.cumsum(t == 2) - 1
        hit = t == 0
        cnt = np.zeros((b.total_roads, 8), np.int64)
        np.add.at(cnt, (road_of_word[hit], layer[hit]), 1)
        assert np.array_equal(cnt[:, :6], b.n_hits)


# --------------------------------------------------------------------------- closed form
def test_linear_tracks_fit_back_to_truth():
    consts = synth.make_constants(64)
    b = synth.make_tracks_batch(consts, 400, seed=3, mode="linear", sigma_scale=0.0)
    cfg = oracle.config(consts.oshift, consts.qshift, 0xFFFFFFFF, 64, 5, 64)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q, cfg)
    assert key == oracle.KEY_OK
    truth = synth.truth_in_output_units(consts, b)
    p = rec[:, 3:].view(np.int32).astype(np.float64)
    F63 = consts.F[b.sector, 63].astype(np.float64)                 # [R,6,6]
    # error budget per row, in output LSB: coordinate rounding (0.5 LSB each),
    # int16 rounding of F (0.5/2^15 per element times x <= 32767) and of q
    # (0.5), and the floor of the final shift (1)
    bound = np.abs(F63[:, :3, :]).sum(axis=2) * 0.5 / 2 ** 15 + 6 * 0.5 * 32767 / 2 ** 15 + 0.5 + 1
    assert np.all(np.abs(p - truth) <= bound), np.max(np.abs(p - truth) / bound)
    chi_bound = np.abs(F63[:, 3:, :]).sum(axis=2) * 0.5 / 2 ** 15 + 6 * 0.5 * 32767 / 2 ** 15 + 0.5 + 1
    assert np.all(rec[:, 2] <= np.sum(np.floor(chi_bound) ** 2, axis=1))
    assert np.all(rec[:, 0] >> 24 == oracle.F_PASS)


def test_smeared_linear_tracks_chi2_is_chi_square_3dof():
    # with Gaussian smearing the chi rows are unit normals before scaling, so
    # chi2 * unit_chi^2 follows a chi-square with 3 degrees of freedom
    consts = synth.make_constants(64)
    b = synth.make_tracks_batch(consts, 6000, seed=4, mode="linear", sigma_scale=1.0)
    cfg = oracle.config(consts.oshift, consts.qshift, 0xFFFFFFFF, 64, 5, 64)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q, cfg)
    assert key == oracle.KEY_OK
    z = rec[:, 2].astype(np.float64) * consts.unit_chi ** 2
    assert abs(z.mean() - 3.0) < 0.15
    assert abs(np.mean(z <= synth.CHI2_Q99_3DOF) - 0.99) < 0.006


def test_helix_tracks_stay_close_to_linear_fit():
    consts = synth.make_constants(64)
    b = synth.make_tracks_batch(consts, 500, seed=5, mode="helix", sigma_scale=0.0)
    cfg = oracle.config(consts.oshift, consts.qshift, 0xFFFFFFFF, 64, 5, 64)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q, cfg)
    assert key == oracle.KEY_OK
    z = rec[:, 2].astype(np.float64) * consts.unit_chi ** 2
    # the exact circle departs from the first-order form by far less than the
    # hit resolution, so noise-free helices have chi2 well inside the 99 % cut
    assert np.all(z < synth.CHI2_Q99_3DOF)


# --------------------------------------------------------------------------- drivers agree
def test_omp_and_road_sample_match_serial_run():
    spec = synth.SPECS["scaled"]
    consts = synth.make_constants(spec.n_sectors)
    b = synth.make_batch(spec, 40, consts)
    cfg = oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors)
    key, rec = oracle.run(b.words, b.event_off, consts.F, consts.q, cfg)
    key2, rec2 = oracle.run(b.words, b.event_off, consts.F, consts.q, cfg, omp=True)
    assert key == key2 == oracle.KEY_OK
    assert np.array_equal(rec, rec2)
    pos = np.flatnonzero((b.words >> 30) == 2)
    sel = np.arange(0, len(pos), 7)
    rec3 = oracle.run_roads(b.words, pos[sel], consts.F, consts.q, cfg)
    assert np.array_equal(rec3, rec[sel])
    assert rec.shape == (b.total_roads, 6)


# --------------------------------------------------------------------------- track-trigger pairs
def test_xft_pairs_enumeration_against_big_integers():
    """With xft_pairs the combinations run over layers 0..4 (layer 0 most
    significant, layer 4 fastest) and layer 5 takes layer 4's hit: every y of
    every combination against Python integers, the count against the closed
    form prod_{l<5} max(n_l, 1), and the best record against exhaustion."""
    rng = np.random.default_rng(61)
    S = 2
    F = rng.integers(-32768, 32768, (S, 64, 6, 6)).astype(np.int16)
    q = rng.integers(-32768, 32768, (S, 64, 6)).astype(np.int16)
    for trial in range(200):
        n, hits = random_road(rng, max_hits=3)
        n[5] = n[4]
        hits[5] = rng.integers(0, 32768, int(n[5])).tolist()
        sector = int(rng.integers(0, S))
        cfg = oracle.config(15, 15, 0xFFFFFFFF, 1 << 24, 0, S, xft_pairs=1)
        rec, chi2s, ys = oracle.road(n, hits, sector, 3, F, q, cfg, detail=True)
        mask = sum(1 << l for l in range(6) if n[l] > 0)
        combos = list(itertools.product(*[range(max(int(k), 1)) for k in n[:5]]))
        assert len(chi2s) == len(combos) == int(np.prod(np.maximum(n[:5], 1)))
        best = None
        for c, idx in enumerate(combos):
            i = list(idx) + [idx[4]]
            x = [hits[l][i[l]] if n[l] > 0 else 0 for l in range(6)]
            y_ref, chi_ref = bigint_fit(F[sector, mask].ravel(), q[sector, mask], x, 15, 15)
            assert list(ys[c]) == y_ref and chi2s[c] == chi_ref
            if best is None or chi_ref < best[1]:
                best = (c, chi_ref)
        assert rec[1] == best[0] and rec[2] == best[1]
        # without pairing the same road has n_5 times as many combinations
        cfg0 = oracle.config(15, 15, 0xFFFFFFFF, 1 << 24, 0, S)
        assert len(oracle.road(n, hits, sector, 3, F, q, cfg0, detail=True)[1]) == \
            len(combos) * max(int(n[5]), 1)


def test_xft_unpaired_rule():
    """V11: with xft_pairs a road whose layer-4 and layer-5 hit counts differ is
    reported at the last word of its hit run (code 12); the same words are
    valid without pairing, and the smaller key still wins against other
    rules."""
    ev = ["E:1:3",
          "R:0:1", "H:0:5", "H:1:5", "H:2:5", "H:3:5", "H:4:1", "H:4:2", "H:5:9", "H:5:8",   # paired
          "R:0:2", "H:0:5", "H:4:1", "H:4:2", "H:5:9",                                       # 2 vs 1
          "R:0:3", "H:0:5", "H:1:5"]                                                         # 0 vs 0
    w = tokens_to_words(ev)
    off = np.array([0, len(w)], np.uint64)
    assert oracle.validate(w, off, 1) == oracle.KEY_OK
    assert oracle.decode_key(oracle.validate(w, off, 1, xft_pairs=1)) == (14, oracle.E_XFT_UNPAIRED)
    # the last road of an event is closed by the end of the event
    w2 = tokens_to_words(["E:1:1", "R:0:1", "H:0:5", "H:5:9"])
    assert oracle.decode_key(oracle.validate(w2, np.array([0, 4], np.uint64), 1, xft_pairs=1)) == \
        (3, oracle.E_XFT_UNPAIRED)
    # an earlier violation gives the smaller key; a later one does not
    bad_early = list(ev)
    bad_early[2] = "HX:6:0:5"          # layer 6 at word 2, before the unpaired run ending at 14
    k = oracle.validate(tokens_to_words(bad_early), off, 1, xft_pairs=1)
    assert oracle.decode_key(k) == (2, oracle.E_BAD_LAYER)
    bad_late = list(ev)
    bad_late[16] = "HX:6:0:5"          # word 16, after it
    k = oracle.validate(tokens_to_words(bad_late), off, 1, xft_pairs=1)
    assert oracle.decode_key(k) == (14, oracle.E_XFT_UNPAIRED)
    # a batch through orc_run reports the key and no records
    F = np.zeros((1, 64, 6, 6), np.int16)
    q = np.zeros((1, 64, 6), np.int16)
    key, rec = oracle.run(w, off, F, q, oracle.config(n_sectors=1, min_layers=0, xft_pairs=1))
    assert key == (14 << 8 | oracle.E_XFT_UNPAIRED) and rec is None
    # a long run: V11 would sit at its last word, after the run's 17th hit
    # of one layer (V8), so the smaller key is V8's
    long = ["E:1:1", "R:0:1"] + ["H:4:1"] * 17 + ["H:5:2"] * 2
    wl = tokens_to_words(long)
    k = oracle.validate(wl, np.array([0, len(wl)], np.uint64), 1, xft_pairs=1)
    assert oracle.decode_key(k) == (18, oracle.E_TOO_MANY_HITS)


def test_xft_generated_batches_pair_their_track_trigger_hits():
    spec = synth.SPECS["xft"]
    consts = synth.make_constants(spec.n_sectors)
    b = synth.make_batch(spec, 30, consts)
    assert np.array_equal(b.n_hits[:, 4], b.n_hits[:, 5])
    assert oracle.validate(b.words, b.event_off, spec.n_sectors, xft_pairs=1) == oracle.KEY_OK
    assert oracle.config(xft_pairs=2) and not oracle.lib().orc_config_ok(oracle.config(xft_pairs=2))
