"""Zero-copy ingest: the fused path reading its words and offsets from mapped
host memory, and writing its records there, gives the oracle's records bit
for bit; the allocator refuses bad arguments."""
import numpy as np
import pytest

from svt_testlib import batch_for, cfg_pair, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_mapped_host_allocator_arguments():
    import ctypes
    from paper_1311_0380_gb300 import _native as N
    L = N.load()
    h, d = ctypes.c_void_p(), ctypes.c_void_p()
    BAD_ARG = 1
    assert L.svt_host_alloc(0, ctypes.byref(h), ctypes.byref(d)) == BAD_ARG
    assert L.svt_host_alloc(4096, None, ctypes.byref(d)) == BAD_ARG
    assert L.svt_host_free(None) == BAD_ARG
    assert L.svt_host_alloc(4096, ctypes.byref(h), ctypes.byref(d)) == N.SVT_OK
    assert h.value and d.value and h.value % 256 == 0 and d.value % 256 == 0
    assert L.svt_host_free(h) == N.SVT_OK


@pytest.mark.parametrize("out_in_host", [False, True])
def test_fused_path_reads_and_writes_host_memory_in_place(out_in_host):
    import torch
    from paper_1311_0380_gb300 import _native as N, api
    spec, consts, b = batch_for("scaled", 100)
    cfg, ocfg = cfg_pair(chi2_cut=consts.chi2_cut_99, max_comb=spec.max_comb)
    key, rec = oracle_run(b.words, b.event_off, consts.F, consts.q, ocfg)
    dc = api.DeviceConstants.from_numpy(consts.F, consts.q, cfg)
    nw, ne, R = len(b.words), b.n_events, b.total_roads
    fp = api.FusedPath(nw, ne, R, dc)
    w_bytes = (4 * nw + 255) // 256 * 256
    m = api.MappedHost(w_bytes + 8 * (ne + 1) + 24 * R)
    m.view(np.uint32, 0, nw)[:] = b.words
    m.view(np.uint64, w_bytes, ne + 1)[:] = b.event_off
    out_off = w_bytes + 8 * (ne + 1)
    out = m.device(out_off) if out_in_host else fp.out
    for _ in range(2):   # twice: nothing of the first call leaks into the second
        api.svt_run(m.device(0), nw, m.device(w_bytes), ne, dc.F, dc.q, cfg, R, out,
                    fp.event_road, fp.counts, fp.status, fp.workspace)
        torch.cuda.synchronize()
        st = int(api.u64(fp.status)[0])
        assert st == key == N.STATUS_OK
        got = (m.view(np.uint32, out_off, 6 * R).reshape(-1, 6).copy() if out_in_host
               else api.u32(fp.out[: 6 * R]).reshape(-1, 6))
        assert np.array_equal(got, rec)
        if out_in_host:
            m.view(np.uint32, out_off, 6 * R)[:] = 0xDEADBEEF
    m.close()
