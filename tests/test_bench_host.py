"""The benchmark's host-side oracle timing (the CPU baseline and the reference arm): one independent oracle room per
host process, started together after a barrier, timed to the slowest process; a process that fails is reported,
never waited on forever."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_oracle_all_cores_two_processes():
    value, elapsed = bench.oracle_all_cores((32, 16, 16), 2, 1, 2)
    assert elapsed > 0
    assert value == pytest.approx(2 * 32 * 16 * 16 * 2 / elapsed / 1e9)


def test_oracle_process_failure_is_reported():
    with pytest.raises(RuntimeError, match="oracle process failed"):
        bench.oracle_all_cores((0, 8, 8), 1, 0, 2)    # nx = 0: the room construction raises


def test_sample_fits_the_budget():
    assert bench.pick_oracle_sample(5, 1e6, 1.0) == (128, 64, 64)
    assert bench.pick_oracle_sample(10**9, 1.0, 1.0) == (32, 16, 16)   # nothing fits: the smallest room
