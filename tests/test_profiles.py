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


def test_work_split_comparison():
    """Schedules that hand the fit kernel the same work units compare equal:
    zero fields mean the defaults, and the split threshold and rows per item
    only count where roads are split at all."""
    import bench
    default = {"warps_per_block": 8, "blocks_per_sm": 0, "rows_per_item": 16,
               "roads_per_chunk": 4, "small_max": 4096, "pair_small": 0}
    zeros = {k: 0 for k in default}
    assert bench.same_work_split(zeros, default, 262144)
    # warps per block and blocks per SM do not change the work units
    assert bench.same_work_split(dict(default, warps_per_block=16, blocks_per_sm=2), default,
                                 262144)
    # with split roads the rows per item and the threshold count ...
    assert not bench.same_work_split(dict(default, rows_per_item=256), default, 262144)
    assert not bench.same_work_split(dict(default, small_max=1024), default, 262144)
    # ... without them (every road within the threshold) they do not
    assert bench.same_work_split(dict(default, rows_per_item=256, small_max=16384), default, 4096)
    assert not bench.same_work_split(dict(default, roads_per_chunk=2), default, 4096)
    assert not bench.same_work_split(dict(default, pair_small=3), default, 4096)
    assert not bench.same_work_split(None, default, 4096)
    # the recorded schedules parse
    assert bench.recorded_schedule()["rows_per_item"] >= 1
    assert bench.recorded_schedule(bench.UNEVEN_NOTE)["roads_per_chunk"] >= 1
