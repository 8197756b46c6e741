"""The continuous-batching server: every event's records are bit-exact with
the oracle whether the event is served alone or in a mix with others, in both
the fused (graph) mode and the plain per-stage mode; a corrupt event fails
alone; the Poisson driver delivers every event."""
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


def mixed_events():
    consts = synth.make_constants(512)
    a = synth.make_batch("scaled", 240, consts)
    b = synth.make_batch("uneven", 24, consts, seed=99)
    events = []
    for bt in (a, b):
        for e in range(bt.n_events):
            events.append(bt.words[int(bt.event_off[e]):int(bt.event_off[e + 1])])
    rng = np.random.default_rng(3)
    rng.shuffle(events)
    off = np.zeros(len(events) + 1, np.uint64)
    off[1:] = np.cumsum([len(x) for x in events])
    return consts, np.concatenate(events).astype(np.uint32), off


def oracle_per_event(words, off, consts, ocfg):
    key, rec = oracle.run(words, off, consts.F, consts.q, ocfg, omp=True)
    assert key == oracle.KEY_OK
    nr = (words[off[:-1].astype(np.int64)] & 0xFFF).astype(np.int64)
    base = np.concatenate([[0], np.cumsum(nr)])
    return [rec[base[e]:base[e + 1]] for e in range(len(nr))], nr


def make_server(consts, mode, **kw):
    from paper_1311_0380_gb300 import api, serve
    cfg = api.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    args = dict(n_slots=4, max_words=1 << 20, max_events=64, max_roads=1 << 15, mode=mode)
    if mode == 1:
        args.update(n_slots=1, max_combs=(1 << 15) * 4096)
    args.update(kw)
    return serve.Server(dc, **args), dc


def collect(srv, n, timeout_polls=20000):
    got = {}
    for _ in range(timeout_polls):
        for r in srv.poll(wait_us=2000):
            got[int(r.tag)] = r
        if len(got) >= n:
            break
    return got


@pytest.mark.parametrize("mode,small", [(0, 0), (1, 0), (0, 4)])
def test_alone_and_in_mix_are_bit_exact(mode, small):
    """small: batches of at most that many events replay the slot's second
    graph (one persistent block per SM, one road per chunk)."""
    from paper_1311_0380_gb300 import api, serve
    consts, words, off = mixed_events()
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    want, nr = oracle_per_event(words, off, consts, ocfg)
    pool = serve.pinned_pool(words)
    kw = {} if not small else dict(sched=api.schedule(8, 0, 16, 1, 4096, 0), small_batch_events=small,
                                   small_blocks_per_sm=1)
    srv, _ = make_server(consts, mode, **kw)
    E = len(nr)
    views = [pool[int(off[e]):int(off[e + 1])] for e in range(E)]
    # in the mix: everything submitted back to back
    dst = [np.zeros((max(int(nr[e]), 1), 6), np.uint32) for e in range(E)]
    for e in range(E):
        assert srv.submit(views[e], e, dst[e]) == 0
    got = collect(srv, E)
    assert len(got) == E
    for e in range(E):
        assert got[e].status == (1 << 64) - 1
        assert np.array_equal(dst[e][: nr[e]], want[e]), e
    st = srv.stats()
    assert st["events_done"] == E and st["batches"] < E   # events were batched together
    # alone: one event in flight at a time
    for e in range(0, E, 7):
        d1 = np.zeros((max(int(nr[e]), 1), 6), np.uint32)
        assert srv.submit(views[e], 10_000 + e, d1) == 0
        r = collect(srv, 1)
        assert r[10_000 + e].status == (1 << 64) - 1
        assert np.array_equal(d1[: nr[e]], want[e])
    srv.close()


def test_corrupt_event_fails_alone():
    from paper_1311_0380_gb300 import serve
    consts, words, off = mixed_events()
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    want, nr = oracle_per_event(words, off, consts, ocfg)
    bad_e = 17
    w2 = words.copy()
    i = int(off[bad_e]) + 3          # a hit word of the event's first road
    assert (w2[i] >> 30) == 0
    w2[i] |= np.uint32(7 << 27)       # layer 7
    bad_key = oracle.validate(w2[int(off[bad_e]):int(off[bad_e + 1])],
                              np.array([0, int(off[bad_e + 1] - off[bad_e])], np.uint64), 512)
    assert bad_key != oracle.KEY_OK
    pool = serve.pinned_pool(w2)
    srv, _ = make_server(consts, 0)
    E = len(nr)
    dst = [np.zeros((max(int(nr[e]), 1), 6), np.uint32) for e in range(E)]
    views = [pool[int(off[e]):int(off[e + 1])] for e in range(E)]
    for e in range(E):
        assert srv.submit(views[e], e, dst[e]) == 0
    got = collect(srv, E)
    assert len(got) == E
    for e in range(E):
        if e == bad_e:
            assert got[e].status == bad_key
        else:
            assert got[e].status == (1 << 64) - 1
            assert np.array_equal(dst[e][: nr[e]], want[e])
    assert srv.stats()["retried_batches"] >= 1
    srv.close()


def test_oversized_event_is_refused_and_queue_bound_applies():
    from paper_1311_0380_gb300 import serve
    consts, words, off = mixed_events()
    pool = serve.pinned_pool(words)
    srv, _ = make_server(consts, 0, max_words=4096, max_queued_words=8192)
    sizes = np.diff(off.astype(np.int64))
    big = int(np.argmax(sizes))
    assert sizes[big] > 4096
    assert srv.submit(pool[int(off[big]):int(off[big + 1])], 0) == 9   # SVT_ERR_OOM
    srv.close()


def test_poisson_driver_delivers_every_event():
    from paper_1311_0380_gb300 import serve
    consts, words, off = mixed_events()
    pool = serve.pinned_pool(words)
    srv, _ = make_server(consts, 0)
    lat, wall = srv.bench_poisson(pool, off, rate_hz=20000.0, n_events=3000, seed=5)
    assert np.all(lat != np.uint64(2 ** 64 - 1))
    assert np.all(lat > 0) and wall > 0
    assert srv.stats()["events_done"] == 3000
    srv.close()


def test_poisson_stream_at_30khz_matches_oracle():
    """20,000 events shaped like the uneven workload arrive as a Poisson stream
    at 30 kHz through the server in its benchmark configuration; every served
    event's records equal the oracle's for that event."""
    from paper_1311_0380_gb300 import api, serve
    consts = synth.make_constants(512)
    pool_b = synth.make_batch("uneven", 384, consts, seed=synth.BASE_SEED + 40)
    ocfg = oracle.config(15, 15, consts.chi2_cut_99, 4096, 5, 512)
    want, nr = oracle_per_event(pool_b.words, pool_b.event_off, consts, ocfg)
    pool = serve.pinned_pool(pool_b.words)
    srv, _ = make_server(consts, 0, max_words=1 << 22, max_events=256, max_roads=1 << 17,
                         sched=api.schedule(8, 0, 16, 1, 4096, 0), small_batch_events=4,
                         small_blocks_per_sm=1)
    n = 20000
    k = np.arange(n) % len(nr)
    rec_off = np.zeros(n + 1, np.uint64)
    rec_off[1:] = np.cumsum(nr[k])
    rec = np.full((int(rec_off[-1]) + 1, 6), 0xDEADBEEF, np.uint32)
    lat, wall = srv.bench_poisson(pool, pool_b.event_off, 30e3, n, seed=11, records=rec,
                                  rec_off=rec_off)
    assert np.all(lat != np.uint64(2 ** 64 - 1)) and wall > 0
    expect = np.concatenate([want[i] for i in k])
    assert np.array_equal(rec[:-1], expect)
    assert srv.stats()["events_failed"] == 0
    srv.close()


def test_slots_overlap_on_the_device():
    """Events submitted back to back are spread over the slots, and the traced
    device intervals (first copy in to last copy out) of batches in different
    slots overlap: their work is in flight on the GPU at the same time."""
    from paper_1311_0380_gb300 import serve
    consts, words, off = mixed_events()
    pool = serve.pinned_pool(words)
    srv, _ = make_server(consts, 0, max_events=4)
    srv.trace_start(4096)
    E = len(off) - 1
    for e in range(E):
        assert srv.submit(pool[int(off[e]):int(off[e + 1])], e) == 0
    got = collect(srv, E)
    assert len(got) == E
    tr = srv.trace_stop()
    assert len(tr) == srv.stats()["batches"] and len(set(tr["slot"].tolist())) > 1
    assert np.all(tr["dev_end_us"] >= tr["dev_start_us"]) and np.all(tr["dev_start_us"] >= 0)
    assert serve.overlap_fraction(tr) > 0.5
    srv.close()
