"""The bench's roofline `traffic` comes from a committed ncu summary: the
summary of the dominant kernel on the default workload must parse, and its
DRAM bytes per working launch must sit at or above the algorithmic bytes it
quotes (padding and re-reads only add traffic) and within 2x of them."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sweep_traffic_summary_parses():
    tr = bench._ncu_traffic("precond_sweep", "beam_halo_1e7_depth10")
    assert tr is not None and tr["file"].startswith("profiles/")
    assert tr["algorithmic_bytes_per_working_launch"] <= tr["bytes_per_launch"]
    assert tr["bytes_per_launch"] <= 2.0 * tr["algorithmic_bytes_per_working_launch"]


def test_unknown_kernel_has_no_traffic():
    assert bench._ncu_traffic("precond_sweep", "no_such_workload") is None
