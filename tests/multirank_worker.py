"""Worker for tests/test_multirank.py: run under torchrun with the gloo backend.

Checks the benchmark's multi-rank plumbing on CPU: every rank reports its own
units and time; the job value is the sum of units over the slowest rank's time.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def main():
    d = bench.Dist(backend="gloo")
    assert d.world == int(os.environ["WORLD_SIZE"]) and d.world >= 2
    units = 1000.0 * (d.rank + 1)       # rank r processed 1000 (r+1) edges
    ms = 10.0 * (d.rank + 1)            # in 10 (r+1) ms
    value, ms_max = bench.aggregate(units, ms, d)
    total = sum(1000.0 * (r + 1) for r in range(d.world))
    assert ms_max == 10.0 * d.world, ms_max
    assert abs(value - total / (ms_max * 1e-3)) < 1e-6, value
    d.barrier()
    if d.rank == 0:
        print(json.dumps({"ok": True, "world": d.world, "value": value}), flush=True)
    d.close()


if __name__ == "__main__":
    main()
