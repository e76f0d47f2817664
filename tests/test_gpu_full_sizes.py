"""Parity with the oracle at the sizes the product path runs.

* The bench's whole step on the QFT workload (n = 20): the small-frame prefix
  and the grid program (or the grid program alone), then the measurement of
  qubit 0 -- the cofactor of the 2^19-element frame into 2^20 children, merged
  pairwise -- and one amplitude, each compared with the oracle running the same
  step.
* The Cuccaro ripple-carry adder at its stated size (16-bit registers, 34
  qubits) on seeded basis inputs: frame and tableau against the oracle, output
  against a + b mod 2^17; the 7-bit adder on the equal superposition sampled
  qubit by qubit, every measurement's probabilities against the oracle's.
* Frames of 16 and 8 words per phase vector (n = 1000, 300) with more than
  4096 elements: a Clifford scramble, T gates on fresh |+> qubits and on
  scrambled ones, more Clifford gates on the grown frame and a measurement,
  with the low-rank forms of the maps on and off.

Tableau and phase vectors bit for bit; amplitudes and probabilities within
1e-10, the global phase included (Def. 1, Sec. III-IV, Sec. VI).
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.gpu
TOL = 1e-10
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    assert gr == orr, (gr, orr)
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz), "tableau differs"
    gs, ga = g.frame()
    os_, oa = o.frame()
    assert gs.shape == os_.shape, (gs.shape, os_.shape)
    assert np.array_equal(gs, os_), "phase vectors differ"
    if len(ga):
        err = float(np.max(np.abs(ga - oa)))
        assert err <= tol, err
    return len(gs)


def _bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    return bench


def _oracle_plan(n, plan):
    o = oracle.FrameOracle(n)
    for op in plan:
        if op[0] == "C":
            o.apply_clifford(op[1])
        else:
            o.apply_nonclifford(op[1], op[2], op[3], op[4])
            o.coalesce(1e-12)
    return o


@pytest.mark.parametrize("prefix", [1024, 0])
def test_bench_step_vs_oracle(sfm, prefix):
    """The bench's step, record for record: program kernels over the QFT, then
    measure(0, -1) through the per-op path and one amplitude."""
    import torch
    bench = _bench()
    n = bench.N_QUBITS
    x, plan, y = bench.build_plan(n, 0)
    recs, starts = bench.plan_records(sfm, plan)
    d_all = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
    consumed = torch.zeros(1, dtype=torch.int64, device="cuda")
    f = sfm.Frame(n, bench.MAX_ELEMS)
    m = 0
    if prefix:
        f.apply_program_device(d_all.data_ptr(), len(recs), bench.DROP_EPS, consumed.data_ptr(), 0, prefix)
        f.sync()
        m = int(consumed.item())
        assert 0 < m < len(recs)
    f.apply_program_grid_device(d_all.data_ptr() + recs.itemsize * m, len(recs) - m, bench.DROP_EPS,
                                consumed.data_ptr())
    f.sync()
    assert m + int(consumed.item()) == len(recs)
    o = _oracle_plan(n, plan)
    assert frames_equal(f, o) == 1 << 19
    gp = f.measure(0, -1)
    op = o.measure(0, -1)
    assert abs(gp[0] - op[0]) <= TOL and abs(gp[1] - op[1]) <= TOL
    # the cofactor splits each of the 2^19 elements in two; sigma and sigma ^ u_q
    # share their children, so the 2^20 children merge into 2^19 elements
    assert frames_equal(f, o) == 1 << 19
    ga, oa = f.amplitude(y), o.amplitude(y)
    assert abs(ga - oa) <= TOL
    assert abs(ga - c.qft_expected_amplitude(n, x, y)) <= TOL
    f.close()


def test_cuccaro_16bit_basis_inputs(sfm):
    """34 qubits: a_0..a_15, b_0..b_15, ancilla and carry; 16 seeded inputs."""
    nb = 16
    nq = 2 * nb + 2
    rng = c.rng_for(16)
    for _ in range(16):
        av, bv = int(rng.integers(1 << nb)), int(rng.integers(1 << nb))
        ops = c.cuccaro(nb, False, av, bv)
        g = sfm.Frame(nq, 1 << 12)
        o = oracle.FrameOracle(nq)
        c.run(g, ops)
        c.run(o, ops)
        assert frames_equal(g, o) == 1
        out = c.cuccaro_reference(nb, av, bv)
        anc, a, b, z = c.cuccaro_layout(nb)
        s = sum(((out >> b[i]) & 1) << i for i in range(nb)) + (((out >> z) & 1) << nb)
        assert s == (av + bv) % (1 << (nb + 1))
        assert abs(g.amplitude(out) - 1) <= TOL
        g.close()


@pytest.mark.parametrize("seed", range(4))
def test_cuccaro_7bit_superposition_sampled_vs_oracle(sfm, seed):
    """16 qubits (peak frame 2^16): every qubit measured in turn with a seeded
    draw; each probability pair equals the oracle's, the outcomes agree, the
    frames agree after the last collapse, and the sampled output adds up."""
    nb = 7
    nq = 2 * nb + 2
    ops = c.cuccaro(nb, True)
    g = sfm.Frame(nq, 1 << 18)
    o = oracle.FrameOracle(nq)
    c.run(g, ops)
    c.run(o, ops)
    frames_equal(g, o)
    sample = c.cuccaro_sample_ops(nb, seed)
    rg = c.run(g, sample)
    ro = c.run(o, sample)
    for a, b in zip(rg, ro):
        assert a[0] == b[0] and a[3] == b[3]
        assert abs(a[1] - b[1]) <= TOL and abs(a[2] - b[2]) <= TOL
    frames_equal(g, o)
    out = sum(r[3] << r[0] for r in rg)
    anc, a, b, z = c.cuccaro_layout(nb)
    av = sum(((out >> a[i]) & 1) << i for i in range(nb))
    sv = sum(((out >> b[i]) & 1) << i for i in range(nb)) + (((out >> z) & 1) << nb)
    assert (out >> anc) & 1 == 0 and 0 <= sv - av < (1 << nb)
    g.close()


def _random_qubits(x, n):
    """Qubits whose Z anticommutes with some row of M (an X or Y literal)."""
    return [q for q in range(n) if ((x[:, q // 64] >> np.uint64(q % 64)) & np.uint64(1)).any()]


@pytest.mark.parametrize("n,seed,lowrank", [(1000, 0, True), (1000, 1, True), (1000, 0, False), (300, 2, True),
                                             (300, 2, False)])
def test_wide_frame_above_4096_elements(sfm, n, seed, lowrank):
    """n = 1000 (16 words per phase vector) and n = 300 (8 words): 300 random
    Clifford gates on the first n - 12 qubits, H and T on the 12 untouched ones
    (4096 elements), T and T-dagger on two scrambled random qubits (masks across
    many words, 16384 elements), a batch of three Clifford gates on the grown
    frame and a measurement of a fresh qubit with collapse.  With the low-rank
    forms on, the three-gate batch and the measurement must take them (their
    ranks are read back); off, the per-bit forms run; both match the oracle."""
    g = sfm.Frame(n, 1 << 16)
    g.set_lowrank(lowrank)
    o = oracle.FrameOracle(n)
    scr = c.random_clifford(n - 12, 300, 100 + seed)
    c.run(g, scr)
    c.run(o, scr)
    ops = [("C", c.H, q, 0) for q in range(n - 12, n)]
    for q in range(n - 12, n):
        ops += [("N", c.T if q % 2 else c.TDG, q, 0, 0.0), ("K",)]
    c.run(g, ops)
    c.run(o, ops)
    assert frames_equal(g, o) == 4096
    x, _, _ = o.tableau()
    rq = _random_qubits(x, n - 12)
    assert len(rq) >= 6
    pick = [rq[int(i)] for i in c.rng_for(7 + seed).choice(len(rq), size=5, replace=False)]
    ops = [("N", c.T, pick[0], 0, 0.0), ("K",), ("N", c.TDG, pick[1], 0, 0.0), ("K",)]
    c.run(g, ops)
    c.run(o, ops)
    k = frames_equal(g, o)
    assert k > 4096
    ops = [("C", c.H, pick[2], 0), ("C", c.CNOT, pick[3], n - 1), ("C", c.S, pick[4], 0), ("M", n - 3, 0.3)]
    rg = c.run(g, ops)
    ro = c.run(o, ops)
    ranks = g.lowrank_ranks()
    if lowrank:
        assert all(0 <= r <= 16 for r in ranks), ranks
    else:
        assert ranks == (-1, -1, -1), ranks
    assert rg[0][3] == ro[0][3]
    assert abs(rg[0][1] - ro[0][1]) <= TOL and abs(rg[0][2] - ro[0][2]) <= TOL
    assert frames_equal(g, o) > 2048
    g.close()


def test_wide_scramble_batch_takes_the_per_bit_form(sfm):
    """One batch of 300 random Clifford gates on a grown n = 1000 frame: the
    map's rank exceeds the low-rank limit, the per-bit kernel applies it, and
    the frame still matches the oracle."""
    n = 1000
    g = sfm.Frame(n, 1 << 12)
    o = oracle.FrameOracle(n)
    ops = [("C", c.H, q, 0) for q in range(8)]
    for q in range(8):
        ops += [("N", c.T, q, 0, 0.0), ("K",)]
    ops += c.random_clifford(n, 300, 5)
    c.run(g, ops)
    c.run(o, ops)
    assert g.lowrank_ranks()[0] == -1
    assert frames_equal(g, o) == 256
    g.close()
