"""The figures bench.py takes from the committed ncu summaries (instructions
per combination of the fit kernel, its DRAM traffic per launch) are keyed to
the SHA-256 of the fit kernel's sources; the bench reports the issue
fraction and the traffic only while they match.  This fails as soon as the
kernel source changes without the summaries being captured again, so that
the bench line never loses them unnoticed (no GPU needed)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_recorded_fit_kernel_figures_match_the_current_source():
    import bench
    assert bench.recorded_profile("warp_instructions_per_fit") is not None, (
        "profiles/fit_persistent_scaled3000.md: kernel_sha differs from "
        + bench.file_sha(bench.FIT_KERNEL_SRC))
    assert bench.recorded_traffic() is not None
    assert bench.recorded_profile("warp_instructions_per_fit_uneven",
                                  bench.UNEVEN_NOTE) is not None, (
        "profiles/fit_persistent_uneven512.md: kernel_sha differs from "
        + bench.file_sha(bench.FIT_KERNEL_SRC))


def test_recorded_figures_are_plausible():
    import bench
    ipf = bench.recorded_profile("warp_instructions_per_fit")
    ipf_uneven = bench.recorded_profile("warp_instructions_per_fit_uneven", bench.UNEVEN_NOTE)
    traffic = bench.recorded_traffic()
    # at least the inner loop's share (about 18 warp instructions per 32
    # combinations) and no more than a few per combination
    assert 0.5 < ipf_uneven < ipf < 4.0
    # the kernel reads the words and descriptors once: tens of MB, not GB
    assert 1e7 < traffic < 1e8
