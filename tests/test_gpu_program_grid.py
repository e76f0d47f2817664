"""sf_apply_program_grid: Clifford and diagonal records in one cooperative
launch over the whole GPU, up to the first measurement or conditional record.
The frames must equal the oracle's (tableau and phase vectors bit for bit,
amplitudes within 1e-10) wherever the program stops; bad records, the frame
capacity and the qubit limit are rejected, and the handle keeps working."""
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


def clifford_diag_circuit(n, seed, length=300, p_diag=0.12, with_meas=False):
    """Random Clifford gates with merged diagonal gates (T, T-dagger, phase,
    controlled phase) mixed in; optionally one measurement with its draw."""
    g = c.rng_for(seed)
    ops = []
    kinds = tuple(range(9)) if n > 1 else (0, 1, 2, 3, 4, 5)
    meas_at = length // 2 if with_meas else -1
    for i, op in enumerate(c.random_clifford(n, length, seed=seed, kinds=kinds)):
        ops.append(op)
        if i == meas_at:
            ops.append(("M", int(g.integers(n)), float(g.random())))
        r = g.random()
        if r < p_diag:
            kind = int(g.integers(3))
            ops += [("N", kind, int(g.integers(n)), 0, float(g.uniform(-3, 3))), ("K",)]
        elif r < 1.5 * p_diag and n > 1:
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            ops += [("N", c.CPHASE, a, b, float(g.uniform(-3, 3))), ("K",)]
    return ops


def run_grid_then_ops(sfm, n, ops, cap):
    f = sfm.Frame(n, cap)
    i = f.apply_program_grid(ops)
    c.run(f, ops[i:])
    return f, i


@pytest.mark.parametrize("n,seed", [(1, 0), (5, 1), (12, 2), (20, 3), (33, 4), (63, 5)])
def test_grid_program_matches_oracle(sfm, n, seed):
    ops = clifford_diag_circuit(n, 1000 * n + seed)
    f, i = run_grid_then_ops(sfm, n, ops, 1 << 18)
    assert i == len(ops)
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid_program_stops_at_measurement(sfm, seed):
    """The program ends before the measurement; the per-op calls finish the
    circuit with the same outcomes and frames as the oracle."""
    n = 14
    ops = clifford_diag_circuit(n, 77 + seed, with_meas=True)
    f, i = run_grid_then_ops(sfm, n, ops, 1 << 18)
    assert ops[i][0] == "M"
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


@pytest.mark.parametrize("prefix", [False, True])
def test_qft_n20_grid(sfm, prefix):
    """The headline workload: the whole QFT in the grid program, or its small-
    frame prefix in the single-CTA program and the rest in the grid program."""
    x, ops = c.qft_random_input(20, seed=0)
    f = sfm.Frame(20, 1 << 21)
    i = f.apply_program(ops, max_frame=2048)[0] if prefix else 0
    j = f.apply_program_grid(ops[i:])
    assert i + j == len(ops)
    o = oracle.FrameOracle(20)
    c.run(o, ops)
    assert frames_equal(f, o) == 1 << 19
    for y in c.rng_for(5).integers(1 << 20, size=3):
        assert abs(f.amplitude(int(y)) - c.qft_expected_amplitude(20, x, int(y))) <= TOL
    f.close()


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_qft_n16_grid_with_cancellations(sfm, seed):
    """QFT inputs whose frames lose elements to exact cancellation: the
    in-place runs must drop them like the per-gate merges do."""
    x, ops = c.qft_random_input(16, seed=seed)
    f = sfm.Frame(16, 1 << 18)
    assert f.apply_program_grid(ops) == len(ops)
    o = oracle.FrameOracle(16)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


def test_grid_in_place_runs_and_compaction(sfm):
    """T then T-dagger on the same qubits (the second merge of each pair runs
    in place and cancels half the frame, which is then compacted), phase gates
    on qubits in the stabilizer group (in place, no partners), and controlled
    phases sharing a mask."""
    n = 9
    ops = [("C", c.H, q, 0) for q in range(n)]
    for q in (0, 3, 5):
        ops += [("N", c.T, q, 0, 0.0), ("K",), ("N", c.PHASE, q, 0, 0.7), ("K",), ("N", c.TDG, q, 0, 0.0), ("K",),
                ("N", c.PHASE, q, 0, -0.7), ("K",)]
    ops += [("C", c.H, 1, 0), ("N", c.PHASE, 1, 0, 0.3), ("K",), ("N", c.CPHASE, 1, 2, 1.1), ("K",),
            ("C", c.X, 4, 0), ("C", c.H, 4, 0), ("C", c.H, 4, 0)]
    for m in (5, 6, 7, 8):
        ops += [("N", c.CPHASE, 4, m, 0.4 * m), ("K",)]
    f = sfm.Frame(n, 1 << 12)
    assert f.apply_program_grid(ops) == len(ops)
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


def test_grid_program_twice_and_only_cliffords(sfm):
    """Consecutive launches on one handle (the barrier state carries over), a
    program of Clifford records only, and an odd and even number of merges."""
    n = 10
    ops = clifford_diag_circuit(n, 4242, length=120)
    f = sfm.Frame(n, 1 << 16)
    h = len(ops) // 2
    while h < len(ops) and ops[h][0] == "K":
        h += 1
    assert f.apply_program_grid(ops[:h]) == h
    assert f.apply_program_grid(ops[h:]) == len(ops) - h
    cl = [op for op in c.random_clifford(n, 50, seed=9)]
    assert f.apply_program_grid(cl) == len(cl)
    one = [("N", c.T, 3, 0, 0.0), ("K",)]
    assert f.apply_program_grid(one) == 2
    o = oracle.FrameOracle(n)
    c.run(o, ops + cl + one)
    frames_equal(f, o)
    f.close()


def test_grid_program_errors(sfm):
    import torch
    n = 8
    good = [("C", c.H, q, 0) for q in range(n)] + [("N", c.T, 0, 0, 0.0), ("K",)]
    recs, _ = sfm.encode_program([good])
    # a bad record: SF_EINVAL, nothing applied
    bad = recs.copy()
    bad["q0"][2] = n
    d_bad = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    f = sfm.Frame(n, 64)
    f.apply_clifford([(c.H, 1, 0)])
    f.apply_program_grid_device(d_bad.data_ptr(), len(bad))
    with pytest.raises(sfm.SFError) as e:
        f.sync()
    assert e.value.code == sfm.SF_EINVAL
    o = oracle.FrameOracle(n)
    o.apply_clifford([(c.H, 1, 0)])
    frames_equal(f, o)
    # the handle works after the error
    assert f.apply_program_grid(good) == len(good)
    c.run(o, good)
    frames_equal(f, o)
    # capacity: T gates on fresh |+> qubits double the frame; 8 elements max
    g = sfm.Frame(n, 8)
    grow = [("C", c.H, q, 0) for q in range(n)]
    for q in range(5):
        grow += [("N", c.T, q, 0, 0.0), ("K",)]
    recs2, _ = sfm.encode_program([grow])
    d2 = torch.from_numpy(recs2.view(np.uint8).copy()).cuda()
    g.apply_program_grid_device(d2.data_ptr(), len(recs2))
    with pytest.raises(sfm.SFError) as e:
        g.sync()
    assert e.value.code == sfm.SF_ECAPACITY
    o2 = oracle.FrameOracle(n)
    c.run(o2, grow[:n + 6])  # the three merges that fit
    frames_equal(g, o2)
    # more than 63 qubits is rejected
    w = sfm.Frame(64, 16)
    with pytest.raises(sfm.SFError):
        w.apply_program_grid_device(d2.data_ptr(), len(recs2))
    for x in (f, g, w):
        x.close()


def _forget_hull(f):
    """A diagonal gate of angle 0 (the identity) through the per-op path: the
    state is unchanged, and the handle no longer vouches for the frame's hull,
    so the grid program that follows merges every branch through the index."""
    f.apply_nonclifford_coalesce(c.PHASE, 0, 0, 0.0, 1e-12)


@pytest.mark.parametrize("n,seed", [(6, 10), (12, 11), (20, 12), (40, 13), (63, 14)])
@pytest.mark.parametrize("known", [True, False])
def test_grid_program_with_and_without_hull(sfm, n, seed, known):
    """Branches along directions new to the frame run as in-place passes when the
    hull is known (from the reset) and as index merges when it is not; both
    equal the oracle."""
    ops = clifford_diag_circuit(n, 5000 + seed, length=400, p_diag=0.2)
    f = sfm.Frame(n, 1 << 18)
    if not known:
        _forget_hull(f)
    i = f.apply_program_grid(ops)
    assert i == len(ops)
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


@pytest.mark.parametrize("seed", range(6))
def test_grid_program_stage_passes(sfm, seed):
    """Stages that branch along new directions, runs that keep the pairs (found
    by position), uniform and partial drops, more stages than one plan batch
    holds; against the oracle."""
    n = 16
    ops = c.stage_circuit(n, 700 + seed, stages=14, per_stage=40)
    f = sfm.Frame(n, 1 << 18)
    assert f.apply_program_grid(ops) == len(ops)
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


@pytest.mark.parametrize("one_cta", [False, True])
@pytest.mark.parametrize("n,seed", [(10, 0), (30, 1), (63, 2), (70, 3), (200, 4)])
def test_run_program_from_host_records(sfm, n, seed, one_cta):
    """sf_run_program: the whole circuit (Clifford gates, diagonal gates,
    measurements with draws, conditional gates) from host records, through the
    grid program or, with SF_RUN_ONE_CTA, the single-CTA program (n <= 63),
    or the per-op calls; against the oracle."""
    ops = clifford_diag_circuit(n, 9000 + seed, length=250, with_meas=True)
    ops += [("M", (3 * seed) % n, 0.37)]
    f = sfm.Frame(n, 1 << 16)
    bits, nm = f.run_program(ops, one_cta=one_cta)
    o = oracle.FrameOracle(n)
    res = c.run(o, ops)
    assert nm == len(res)
    assert bits == sum(r[3] << i for i, r in enumerate(res))
    frames_equal(f, o)
    f.close()


def test_run_program_conditional_gates(sfm):
    """Conditional Clifford gates after two measurements, through
    sf_run_program, against the oracle walking the same ops."""
    n = 5
    ops = [("C", c.H, 0, 0), ("C", c.H, 1, 0), ("N", c.T, 0, 0, 0.0), ("K",), ("M", 0, 0.9), ("M", 1, 0.1),
           ("Q", c.X, 2, 0, 0b11), ("Q", c.H, 3, 0, 0b01), ("N", c.T, 3, 0, 0.0), ("K",), ("M", 3, 0.6)]
    for one_cta in (False, True):
        f = sfm.Frame(n, 1 << 10)
        bits, nm = f.run_program(ops, one_cta=one_cta)
        o = oracle.FrameOracle(n)
        res = c.run(o, ops)
        assert nm == 3 and bits == sum(r[3] << i for i, r in enumerate(res))
        frames_equal(f, o)
        f.close()


def test_run_program_one_cta_outgrows_the_single_cta_limit(sfm):
    """SF_RUN_ONE_CTA with a frame that outgrows the single-CTA limit (16384)
    part way: the per-op calls continue with the outcomes so far, and a
    conditional gate after the switch reads a measurement made on one CTA."""
    n = 24
    ops = [("C", c.H, q, 0) for q in range(n)] + [("M", 3, 0.2)]
    for q in range(4, 20):
        ops += [("N", c.T, q, 0, 0.0), ("K",)]
    ops += [("Q", c.X, 0, 0, 0b1), ("N", c.T, 0, 0, 0.0), ("K",), ("M", 5, 0.7)]
    f = sfm.Frame(n, 1 << 18)
    bits, nm = f.run_program(ops, one_cta=True)
    o = oracle.FrameOracle(n)
    res = c.run(o, ops)
    assert nm == 2 and bits == sum(r[3] << i for i, r in enumerate(res))
    assert f.size() > 16384
    frames_equal(f, o)
    f.close()


def test_grid_barrier_timeout_is_reported_and_the_handle_recovers(sfm):
    """A wait limit of zero polls makes the first grid barrier run out: the call
    reports SF_ETIMEOUT at the next synchronising call (every CTA leaves at a
    barrier, none waits without bound), and after a reset with the default
    limit the same program gives the oracle's frame."""
    n = 20
    x, ops = c.qft_random_input(n, 3)
    f = sfm.Frame(n, 1 << 21)
    f.set_wait_limit(0)
    recs, _ = sfm.encode_program([ops])
    import torch
    d_ops = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    f.apply_program_grid_device(d_ops.data_ptr(), len(recs), 1e-12)
    with pytest.raises(sfm.SFError) as ei:
        f.sync()
    assert ei.value.code == sfm.SF_ETIMEOUT
    f.set_wait_limit(sfm.WAIT_LIMIT_DEFAULT)
    f.reset()
    f.apply_program_grid_device(d_ops.data_ptr(), len(recs), 1e-12)
    f.sync()
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()


def test_traced_launch_same_frame_and_ordered_stamps(sfm):
    """A traced grid-program launch (sf_set_trace) gives the same frame as the
    oracle; its phase records and the planning CTAs' per-step stamps
    (sf_grid_program_plan_trace) are in time order: each step's tableau is
    published after it starts, the plan CTA takes it after it is published,
    and the plan CTA's stages follow one another."""
    x, ops = c.qft_random_input(12, seed=3)
    f = sfm.Frame(12, 1 << 13)
    f.set_trace(True)
    assert f.apply_program_grid(ops) == len(ops)
    o = oracle.FrameOracle(12)
    c.run(o, ops)
    assert frames_equal(f, o) == 1 << 11
    tr = f.grid_program_trace().astype(np.int64)
    assert len(tr) >= 12
    starts = tr[:, 1]
    assert np.all(starts > 0) and np.all(np.diff(starts) >= 0)
    assert np.all(tr[:, 2] >= tr[:, 1])
    pt = f.grid_program_plan_trace(64).astype(np.int64)
    steps = [m for m in pt if m[7]]  # steps the plan CTA published
    assert len(steps) >= 11
    for m in steps:
        assert m[0] <= m[1] <= m[2], m
        assert np.all(np.diff(m[2:8]) >= 0), m
    pubs = [int(m[7]) for m in steps]
    assert pubs == sorted(pubs)
    f.set_trace(False)
    f.close()
