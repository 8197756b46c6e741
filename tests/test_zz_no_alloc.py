"""svt_run_noalloc, the entry point for callers that cannot allocate device
memory (a front-end that only gets device pointers from the GPU's owner, a
real-time loop that must not allocate once data taking has started, a host
program without a device allocator): its scratch is a fixed array inside the
library.  Its records, status and counts must equal svt_run's on the same
input, on two calls in a row (the array keeps the previous call's contents),
and its records must equal the oracle's.

Kept in a file of its own that pytest collects last.
"""
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


def _run_both(batch, consts, spec):
    import torch
    from paper_1311_0380_gb300 import api
    cfg = api.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5, spec.n_sectors)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    R = batch.total_roads
    dw, de = api.to_device_u32(batch.words), api.to_device_u64(batch.event_off)
    nw, ne = len(batch.words), batch.n_events
    # existing entry point, caller-allocated workspace
    fp = api.FusedPath(nw, ne, R, dc)
    fp.run(dw, nw, de, ne)
    torch.cuda.synchronize()
    st_ref, rec_ref, cnt_ref = fp.result()
    # entry point without a workspace
    out = torch.full((R * 6,), -1, dtype=torch.int32, device="cuda")
    ev = torch.empty(ne + 1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(4, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int64, device="cuda")
    api.svt_run_noalloc(dw, nw, de, ne, dc.F, dc.q, cfg, R, out, ev, counts, status)
    torch.cuda.synchronize()
    st = int(api.u64(status)[0])
    rec = api.u32(out).reshape(-1, 6)
    return (st_ref, rec_ref, cnt_ref, api.u32(fp.event_road)[: ne + 1]), (st, rec, api.u64(counts), api.u32(ev))


def test_noalloc_matches_svt_run_on_two_calls_in_a_row():
    consts = synth.make_constants(512)
    for name, ne, seed in (("scaled", 400, 11), ("uneven", 6, 12)):
        spec = synth.SPECS[name]
        batch = synth.make_batch(spec, ne, consts, seed=seed)
        ref, got = _run_both(batch, consts, spec)
        assert got[0] == ref[0] == (1 << 64) - 1
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
        assert np.array_equal(got[3], ref[3])
        key, want = oracle.run(batch.words, batch.event_off, consts.F, consts.q,
                               oracle.config(15, 15, consts.chi2_cut_99, spec.max_comb, 5,
                                             spec.n_sectors), omp=True)
        assert key == oracle.KEY_OK and np.array_equal(got[1], want)


def test_noalloc_refuses_a_batch_larger_than_its_scratch():
    import torch
    from paper_1311_0380_gb300 import api, _native
    limit = _native.load().svt_run_noalloc_scratch_bytes()
    assert limit == 32 << 20
    cfg = api.config(n_sectors=512)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    q = torch.zeros(512 * 64 * 6, dtype=torch.int16, device="cuda")
    F = torch.zeros(512 * 64 * 36, dtype=torch.int16, device="cuda")
    # a road capacity whose per-road arrays alone exceed the scratch
    with pytest.raises(_native.SvtError, match="OOM"):
        api.svt_run_noalloc(dummy, 16, off, 1, F, q, cfg, 4_000_000, dummy, dummy, None, off)
