"""bench.py reads the DRAM traffic of the gradient kernel from the committed
ncu summary only while the kernel source matches the profiled one."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_profiled_traffic_parses_summary():
    import bench

    fields = {}
    for line in open(bench.GRAD_PROFILE):
        if ": " in line:
            k, v = line.split(": ", 1)
            fields[k.strip()] = v.strip()
    assert "grad.cu sha256[:16]" in fields and "traffic_bytes_per_launch" in fields
    t = bench.profiled_traffic()
    if fields["grad.cu sha256[:16]"] != bench.grad_source_hash():
        assert t is None
        pytest.skip("gradient kernel changed since its profile")
    n, d = 131072, 2048
    algorithmic = 4.0 * n * d + 4.0 * n + 8.0 * d
    assert algorithmic <= t <= 1.1 * algorithmic
