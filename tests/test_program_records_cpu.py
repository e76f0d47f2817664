"""Host-side pieces of the program entry points (no GPU): the mapping from
applied records back to op indices, and the bench's records of the QFT plan."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1712_03554_gb300 import circuits as c  # noqa: E402
from paper_1712_03554_gb300 import sf  # noqa: E402


def test_ops_consumed_maps_records_to_ops():
    ops = [("C", c.H, 0, 0), ("N", c.T, 0, 0, 0.0), ("K",), ("C", c.S, 1, 0), ("K",), ("M", 0, 0.5),
           ("N", c.CPHASE, 0, 1, 0.3), ("K",)]
    # records: C, N, C, M, N  (a "K" has none; the one after "N" belongs to it)
    assert sf._ops_consumed(ops, 0) == 0
    assert sf._ops_consumed(ops, 1) == 1
    assert sf._ops_consumed(ops, 2) == 3      # the merge's "K" goes with its "N"
    assert sf._ops_consumed(ops, 3) == 5      # a lone "K" after it is skipped too
    assert sf._ops_consumed(ops, 4) == 6
    assert sf._ops_consumed(ops, 5) == len(ops)
    assert sf._ops_consumed(ops, 99) == len(ops)


def test_bench_plan_records_match_the_circuit():
    import bench
    x, plan, y = bench.build_plan(8, seed=3)
    recs, starts = bench.plan_records(sf, plan)
    _, ops = c.qft_random_input(8, 3)
    enc, _ = sf.encode_program([ops])
    # the bench's records are the circuit's records: one per gate, diagonal gates merged
    assert len(recs) == len(enc) and starts[-1] == len(recs)
    for field in ("kind", "q0", "q1"):
        assert np.array_equal(recs[field], enc[field]), field
    assert np.allclose(recs["param"], enc["param"])
    # each plan entry starts where the previous one's records end
    sizes = [len(op[1]) if op[0] == "C" else 1 for op in plan]
    assert list(np.diff(starts)) == sizes
