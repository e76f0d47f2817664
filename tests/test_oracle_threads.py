"""The oracle's element-range threading (Sec. V) changes nothing but speed.

Each phase vector is computed by the same code whether its range runs on one
thread or on many, so the frames must be identical (phase vectors bit for bit,
amplitudes exactly); only sums over the frame (probabilities, amplitude
queries) are added in another order.
"""
import numpy as np
import pytest

import oracle
from paper_1712_03554_gb300 import circuits as c


def _run(n, ops, threads, probes):
    prev = oracle.set_threads(threads)
    try:
        o = oracle.FrameOracle(n)
        res = c.run(o, ops)
        sig, amp = o.frame()
        x, z, r = o.tableau()
        amps = [o.amplitude(p) for p in probes]
        return sig, amp, (x, z, r), res, amps
    finally:
        oracle.set_threads(prev)


@pytest.mark.parametrize("n,seed", [(8, 0), (8, 1), (70, 2)])
def test_threaded_oracle_equals_sequential(n, seed):
    ops = c.random_clifford_t(n, 160, 7, seed=seed) + [("M", 1, 0.4), ("M", 5, 0.7)]
    probes = [int(v) for v in c.rng_for(seed + 5).integers(0, 1 << min(n, 62), size=4)]
    s1, a1, t1, r1, p1 = _run(n, ops, 1, probes)
    s8, a8, t8, r8, p8 = _run(n, ops, 8, probes)
    assert len(s1) >= 8
    assert np.array_equal(s1, s8)
    assert np.array_equal(a1, a8)
    for u, v in zip(t1[:2], t8[:2]):
        assert np.array_equal(u, v)
    assert t1[2] == t8[2]
    for u, v in zip(r1, r8):
        assert u[0] == v[0] and abs(u[1] - v[1]) <= 1e-12
    assert max(abs(u - v) for u, v in zip(p1, p8)) <= 1e-13


def test_qft_threaded_equals_sequential():
    x, ops = c.qft_random_input(12, 3)
    s1, a1, _, _, _ = _run(12, ops, 1, [])
    s4, a4, _, _, _ = _run(12, ops, 4, [])
    assert len(s1) >= 64
    assert np.array_equal(s1, s4) and np.array_equal(a1, a4)
