"""svt_int_peak: the measured integer throughput the fit kernel's rooflines use."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_int_peak_is_plausible_and_checks_its_arguments():
    from paper_1311_0380_gb300 import api, _native as N
    sms = N.load().svt_device_sm_count(0)
    ops = {}
    for mode in (0, 1, 2):
        v, sec = api.int_peak(mode, 1 << 12)
        assert sec > 0
        ops[mode] = v
        # at most 128 int32 lanes per SM per cycle, at a clock below 3 GHz
        assert 0 < v < sms * 128 * 3.0e9, (mode, v)
    # both pipes together carry at least as much as either alone
    assert ops[2] > 0.9 * max(ops[0], ops[1])
    for bad in ((3, 16), (0, 0)):
        with pytest.raises(RuntimeError, match="BAD_ARG"):
            api.int_peak(*bad)
