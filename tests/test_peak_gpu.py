"""svt_pipe_peak: the measured arithmetic throughput beside the fit kernel's rooflines."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_pipe_peak_is_plausible_and_checks_its_arguments():
    from paper_1311_0380_gb300 import api, _native as N
    sms = N.load().svt_device_sm_count(0)
    ops = {}
    for mode in (0, 1, 2, 3):
        v, sec = api.pipe_peak(mode, 1 << 12)
        assert sec > 0
        ops[mode] = v
        # at most 128 lanes per SM per cycle, at a clock below 3 GHz
        assert 0 < v < sms * 128 * 3.0e9, (mode, v)
    # both integer rings together carry at least as much as either alone, and
    # the fp32 stream issues at least as fast as the integer ones
    assert ops[2] > 0.9 * max(ops[0], ops[1])
    assert ops[3] > 0.9 * ops[2]
    for bad in ((4, 16), (0, 0)):
        with pytest.raises(RuntimeError, match="BAD_ARG"):
            api.pipe_peak(*bad)
