"""sf_apply_program: a handle's program in one single-CTA launch while the frame
is small, then the per-op calls.  The frames must equal the oracle's (tableau
and phase vectors bit for bit, amplitudes within 1e-10) wherever the program
stops; bad records and the qubit limit are rejected with the frame intact."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def sfm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1712_03554_gb300 import sf
    sf.load()
    return sf


def frames_equal(g, o, tol=TOL):
    gx, gz, gr = g.tableau()
    ox, oz, orr = o.tableau()
    assert gr == orr
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz), "tableau differs"
    gs, ga = g.frame()
    os_, oa = o.frame()
    assert np.array_equal(gs, os_), "phase vectors differ"
    if len(ga):
        assert np.max(np.abs(ga - oa)) <= tol
    return len(gs)


def run_program_then_ops(sfm, n, ops, cap, split=None, max_frame=0):
    """The program on ops[:split] (all of ops if split is None, stopping where
    the frame outgrows the program's frame limit), then the per-op calls."""
    f = sfm.Frame(n, cap)
    head = ops if split is None else ops[:split]
    i, bits, nm = f.apply_program(head, max_frame=max_frame)
    res = c.run(f, ops[i:], outcome_bits=bits, n_drawn=nm)
    for m, r in enumerate(res):
        bits |= r[3] << (nm + m)
    return f, i, bits


def mixed_circuit(n, seed, length=300):
    g = c.rng_for(seed)
    ops = []
    n_meas = 0
    for op in c.random_clifford(n, length, seed=seed, kinds=tuple(range(9)) if n > 1 else (0, 1, 2, 3, 4, 5)):
        ops.append(op)
        r = g.random()
        if r < 0.04:
            ops += [("N", int(g.integers(3)), int(g.integers(n)), 0, float(g.uniform(-3, 3))), ("K",)]
        elif r < 0.06 and n > 1:
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            ops += [("N", c.CPHASE, a, b, float(g.uniform(-3, 3))), ("K",)]
        elif r < 0.08 and n_meas < 60:
            ops.append(("M", int(g.integers(n)), float(g.random())))
            n_meas += 1
        elif r < 0.10 and n_meas:
            ops.append(("Q", int(g.integers(6)), int(g.integers(n)), 0, int(g.integers(1, 1 << min(n_meas, 60)))))
    return ops


@pytest.mark.parametrize("n,seed", [(1, 0), (5, 1), (20, 2), (33, 3), (63, 4)])
@pytest.mark.parametrize("where", ["all", "half", "early", "limit"])
def test_program_then_ops_matches_oracle(sfm, n, seed, where):
    """The program on the whole circuit, on its first half, on its first
    fifth, or with a frame limit of 2 elements (it stops at the first branch
    that would pass it), the per-op calls doing the rest with the outcomes so
    far carried into conditional gates: same frames and outcomes as the
    oracle."""
    ops = mixed_circuit(n, 100 * n + seed)
    split = {"all": None, "half": len(ops) // 2, "early": len(ops) // 5, "limit": None}[where]
    if split is not None and split < len(ops) and ops[split][0] == "K":
        split += 1  # keep a diagonal gate with its coalesce
    f, i, bits = run_program_then_ops(sfm, n, ops, 1 << 16, split, max_frame=2 if where == "limit" else 0)
    if where != "limit":
        assert i == (len(ops) if split is None else split)
    o = oracle.FrameOracle(n)
    ores = c.run(o, ops)
    assert bits == sum(r[3] << m for m, r in enumerate(ores))
    frames_equal(f, o)
    f.close()


def test_qft_n20_program_prefix(sfm):
    """The headline workload: the program carries the QFT until the frame
    outgrows the single-CTA limit; the grid kernels finish it."""
    x, ops = c.qft_random_input(20, seed=0)
    f, i, _ = run_program_then_ops(sfm, 20, ops, 1 << 21)
    assert 0 < i < len(ops)
    o = oracle.FrameOracle(20)
    c.run(o, ops)
    assert frames_equal(f, o) == 1 << 19
    y = int(c.rng_for(7).integers(1 << 20))
    assert abs(f.amplitude(y) - c.qft_expected_amplitude(20, x, y)) <= TOL
    f.close()


def test_exact_mode_and_errors(sfm):
    import torch
    # a program that fits: exact mode (no consumed counter) runs it all
    ops = [("C", c.H, q, 0) for q in range(4)] + [x for q in range(4) for x in (("N", c.T, q, 0, 0.0), ("K",))]
    recs, _ = sfm.encode_program([ops])
    d_ops = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    f = sfm.Frame(6, 64)
    f.apply_program_device(d_ops.data_ptr(), len(recs))
    assert f.size() == 16
    o = oracle.FrameOracle(6)
    c.run(o, ops)
    frames_equal(f, o)
    # exact mode past the limit: SF_ECAPACITY, frame = state after the applied records
    g = sfm.Frame(6, 8)
    g.apply_program_device(d_ops.data_ptr(), len(recs))
    with pytest.raises(sfm.SFError) as e:
        g.sync()
    assert e.value.code == sfm.SF_ECAPACITY
    assert g.size() == 8
    # a bad record: SF_EINVAL, nothing applied
    bad = recs.copy()
    bad["q0"][3] = 6
    d_bad = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    h = sfm.Frame(6, 64)
    h.apply_clifford([(c.H, 0, 0)])
    h.apply_program_device(d_bad.data_ptr(), len(bad))
    with pytest.raises(sfm.SFError) as e:
        h.sync()
    assert e.value.code == sfm.SF_EINVAL
    o2 = oracle.FrameOracle(6)
    o2.apply_clifford([(c.H, 0, 0)])
    frames_equal(h, o2)
    # more than 63 qubits is rejected
    w = sfm.Frame(64, 16)
    with pytest.raises(sfm.SFError):
        w.apply_program_device(d_ops.data_ptr(), len(recs))
    for x in (f, g, h, w):
        x.close()


@pytest.mark.parametrize("seed", range(4))
def test_program_stage_circuits(sfm, seed):
    """The single-CTA program on stage circuits (new-direction branches, merges
    whose partners exist, in-place runs over scattered pairs), then the per-op
    calls once the frame outgrows it; against the oracle."""
    n = 14
    ops = c.stage_circuit(n, 5100 + seed, stages=12, per_stage=30)
    f, i, _ = run_program_then_ops(sfm, n, ops, 1 << 18, max_frame=16384)
    assert i > len(ops) // 4
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()
