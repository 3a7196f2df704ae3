"""Host-side pieces of the inputs and the bench (no GPU): box subsets of a
multi-box set, and the bounded particle sets the bench's oracle legs time."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_1606_02738_gb300 import inputs  # noqa: E402


def test_subset_boxes_is_the_boxes_themselves():
    p = inputs.batched(n_boxes=6, n_min=2000, n_max=8000, seed=3)
    q = p.subset_boxes(2, 5)
    assert q.n_boxes == 3 and q.n == p.box_offsets[5] - p.box_offsets[2]
    assert q.box_offsets[0] == 0 and q.box_offsets[-1] == q.n
    for j, b in enumerate(range(2, 5)):
        a, c = p.subset_box(b), q.subset_box(j)
        for k in ("x", "v", "m", "u", "h", "box"):
            assert np.array_equal(getattr(a, k), getattr(c, k)), k


def test_oracle_workload_keeps_small_sets_and_bounds_large_ones(monkeypatch):
    p = inputs.batched(n_boxes=6, n_min=2000, n_max=8000, seed=3)
    q, note = bench.oracle_workload("batched", 1.0, p)
    assert q is p and note == ""
    monkeypatch.setattr(bench, "ORACLE_MAX_N", 2 * int(p.box_offsets[2]))
    assert p.n > bench.ORACLE_MAX_N
    q, note = bench.oracle_workload("batched", 1.0, p)
    # the first boxes up to half the limit: boxes 0 and 1
    assert q.n_boxes == 2 and q.n == p.box_offsets[2] and "first 2" in note
    u = inputs.config(1, 0.25)
    monkeypatch.setattr(bench, "ORACLE_MAX_N", 4000)
    q, note = bench.oracle_workload("uniform", 0.25, u)
    assert q.n == 2000 and "shrunk" in note  # the same recipe at half the limit
