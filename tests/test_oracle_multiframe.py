"""Pins of the multiframe oracle (Sec. IV, COALESCE and the merge of frames
with equal matrices) against what the paper and the mathematics fix: the
paper's worked COALESCE example, the state-vector oracle (a multiframe and the
frame it came from are the same state), the postconditions of the procedure,
closed forms of the Cuccaro adder on basis inputs, and planted mistakes."""
import math

import numpy as np
import pytest

import oracle
from oracle import multiframe as mfo
from paper_1712_03554_gb300 import circuits as c

pytestmark = pytest.mark.filterwarnings("ignore")


def dense_equal(mf, dense, n, tol=1e-10):
    for y in range(1 << n):
        assert abs(mf.amplitude(y) - dense.amplitude(y)) <= tol, y


def rows(x, z):
    return [(int(x[r, 0]), int(z[r, 0])) for r in range(x.shape[0])]


def test_paper_coalesce_example():
    """Sec. IV example: phase vectors 000, 010, 100, 111 over M = {Z1, Z2, Z3}
    (equal amplitudes) pair as <s1, s2> with e = {2} and <s3, s4> with
    e = {2, 3}; F1 is M with column 2 conjugated by H, F2 with column 2
    conjugated by H and columns 2, 3 by CNOT; d = 0, so no P gate."""
    mf = mfo.MultiFrameOracle(3)
    mf.apply_clifford([(c.H, 0, 0), (c.H, 1, 0)])
    F = mf.frames[0]
    F.apply_toffoli_cofactor(0, 1, 2)  # |ab0> -> |ab(a and b)>: the four vectors of the example
    F.coalesce()
    x, z, _ = F.tableau()
    assert rows(x, z) == [(0, 1), (0, 2), (0, 4)]  # M = {Z1, Z2, Z3}
    sig, amp = F.frame()
    # entries (e1 e2 e3) = rows 0, 1, 2: 000, 010, 100, 111
    assert sorted(int(s[0]) for s in sig) == sorted([0b000, 0b010, 0b001, 0b111])
    assert np.allclose(amp, 0.5)
    assert mf.coalesce() == (2, 2)
    d = mf.as_dict()
    # RREF rows (x, z) per qubit bit: F1 = {X2, Z1, Z3}, F2 = {X2 X3, Z1, Z2 Z3}
    f1 = (np.array([[0b010], [0], [0]], np.uint64).tobytes(), np.array([[0], [0b001], [0b100]], np.uint64).tobytes())
    f2 = (np.array([[0b110], [0], [0]], np.uint64).tobytes(), np.array([[0], [0b001], [0b110]], np.uint64).tobytes())
    assert set(d) == {f1, f2}
    # F1 holds |0>|+>|0>, all signs +; F2 holds |1>(|00> + |11>)/sqrt 2: Z1 row negative
    assert list(d[f1]) == [0] and abs(d[f1][0] - 1 / math.sqrt(2)) < 1e-12
    assert list(d[f2]) == [0b010] and abs(d[f2][0b010] - 1 / math.sqrt(2)) < 1e-12


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_phase_pairs_use_p_to_the_d(d):
    """a_r = i^d a_j: the pair becomes (|0> + i^d |1>)/sqrt 2 on the qubit, a
    +-X or +-Y row (P^d H); the state is unchanged."""
    n = 3
    mf = mfo.MultiFrameOracle(n)
    F = mf.frames[0]
    x = np.zeros((n, 1), np.uint64)
    z = np.array([[1], [2], [4]], np.uint64)
    a = 0.6 * np.exp(0.3j)
    F.set_state(x, z, np.array([[0b000], [0b010]], np.uint64), np.array([a, a * 1j ** d]) / math.sqrt(2))
    want = np.zeros(1 << n, complex)
    want[0] = a / math.sqrt(2)
    want[0b010] = a * 1j ** d / math.sqrt(2)
    assert mf.coalesce() == (1, 1)
    for y in range(1 << n):
        assert abs(mf.amplitude(y) - want[y]) <= 1e-12
    (key,) = mf.as_dict()
    xs = np.frombuffer(key[0], np.uint64)
    zs = np.frombuffer(key[1], np.uint64)
    y_row = any(int(xs[r]) == 0b010 and int(zs[r]) == 0b010 for r in range(n))
    assert y_row == (d % 2 == 1)


@pytest.mark.parametrize("seed", range(6))
def test_random_toffoli_circuits_keep_the_state(seed):
    """Random Clifford + Toffoli/controlled-R circuits by cofactors: after every
    non-Clifford gate the multiframe equals the state vector."""
    g = c.rng_for(900 + seed)
    n = int(g.integers(4, 8))
    mf = mfo.MultiFrameOracle(n)
    dense = oracle.DenseOracle(n)
    for step in range(14):
        gates = []
        for _ in range(int(g.integers(1, 5))):
            kind = int(g.choice([c.H, c.S, c.CNOT, c.X]))
            q0 = int(g.integers(n))
            q1 = int((q0 + 1 + g.integers(n - 1)) % n) if kind == c.CNOT else 0
            gates.append((kind, q0, q1))
        mf.apply_clifford(gates)
        dense.apply_clifford(gates)
        a, b, t = (int(v) for v in g.choice(n, size=3, replace=False))
        if step % 3 == 2:
            alpha = float(g.choice([math.pi / 2, math.pi / 4, 0.7]))
            mf.apply_cr_cofactor(a, t, alpha)
            dense.apply_cr_cofactor(a, t, alpha)
        else:
            mf.apply_toffoli_cofactor(a, b, t)
            dense.apply_toffoli_cofactor(a, b, t)
        dense_equal(mf, dense, n)


def test_postconditions_after_coalescing():
    """Every frame is in RREF, no two frames share a matrix, no candidate pair
    is left, and the multiframe holds no more states than one frame would."""
    n = 8
    ops = c.cuccaro(3, superpose=True, toffoli="cofactor", coalesce=False)
    mf = mfo.MultiFrameOracle(n)
    single = oracle.FrameOracle(n)
    c.run(mf, ops)
    c.run(single, ops)
    keys = set()
    for F in mf.frames:
        assert F.is_rref()
        x, z, _ = F.tableau()
        keys.add(x.tobytes() + z.tobytes())
        assert mfo.coalesce_frame(F)[1] == 0
    assert len(keys) == len(mf.frames)
    assert mf.count()[1] < single.size()
    dense = oracle.DenseOracle(n)
    c.run(dense, ops)
    dense_equal(mf, dense, n)


@pytest.mark.parametrize("nb", [1, 2, 3])
def test_cuccaro_superposition_matches_state_vector(nb):
    ops = c.cuccaro(nb, superpose=True, toffoli="cofactor", coalesce=False)
    n = 2 * nb + 2
    mf = mfo.MultiFrameOracle(n)
    dense = oracle.DenseOracle(n)
    c.run(mf, ops)
    c.run(dense, ops)
    dense_equal(mf, dense, n)
    assert mf.count()[1] < 4 ** nb


@pytest.mark.parametrize("nb,a,b", [(3, 5, 6), (4, 9, 11), (5, 31, 1)])
def test_cuccaro_basis_inputs_give_the_sum(nb, a, b):
    """Closed form: on basis inputs the adder's output is one basis state."""
    ops = c.cuccaro(nb, superpose=False, a_val=a, b_val=b, toffoli="cofactor", coalesce=False)
    n = 2 * nb + 2
    mf = mfo.MultiFrameOracle(n)
    c.run(mf, ops)
    want = c.cuccaro_reference(nb, a, b)
    assert abs(mf.amplitude(want) - 1.0) < 1e-12
    assert mf.count() == (1, 1)


def test_planted_mistakes_are_caught(monkeypatch):
    """A wrong P direction or a missing sqrt 2 breaks the comparison with the
    state written out by hand."""
    n = 3
    x = np.zeros((n, 1), np.uint64)
    z = np.array([[1], [2], [4]], np.uint64)
    sig = np.array([[0b000], [0b010], [0b001], [0b111]], np.uint64)
    amps = np.array([0.5, 0.5j, 0.5, -0.5])

    def build():
        mf = mfo.MultiFrameOracle(n)
        mf.frames[0].set_state(x, z, sig, amps)
        return mf

    want = {0: 0.5, 0b010: 0.5j, 0b001: 0.5, 0b111: -0.5}

    def ok(mf):
        return all(abs(mf.amplitude(y) - want.get(y, 0)) <= 1e-12 for y in range(1 << n))

    mf = build()
    mf.coalesce()
    assert ok(mf) and mf.count()[1] == 2
    real_ipow = mfo.i_power
    monkeypatch.setattr(mfo, "i_power", lambda ar, aj, tol=mfo.TOL: (lambda d: None if d is None else (-d) % 4)(
        real_ipow(ar, aj, tol)))
    mf = build()
    mf.coalesce()
    assert not ok(mf)
    monkeypatch.setattr(mfo, "i_power", real_ipow)
    monkeypatch.setattr(mfo.math, "sqrt", lambda v: 1.0)
    mf = build()
    mf.coalesce()
    assert not ok(mf)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_one_coalesce_halves_a_fully_paired_frame(n):
    """Sec. IV: the multiframe COALESCE generates holds half the phase vectors
    of its input when every element has a candidate partner.  H on every
    qubit, P(pi/2) branched on each, H again: one frame of 2^n elements over
    Z_k-rows only, with amplitude ratios that are powers of i."""
    mf = mfo.MultiFrameOracle(n)
    mf.apply_clifford([(c.H, q, 0) for q in range(n)])
    for q in range(n):
        mf.apply_nonclifford_coalesce(c.PHASE, q, 0, math.pi / 2)
    mf.apply_clifford([(c.H, q, 0) for q in range(n)])
    (F,) = mf.frames
    x, z, _ = F.tableau()
    assert len(mfo.zk_rows(x, z)) == n and F.size() == 1 << n
    out, pairs = mfo.coalesce_frame(F)
    assert pairs == 1 << (n - 1)
    assert sum(G.size() for G in out) == 1 << (n - 1)


# ---- the two COALESCE readings on the Cuccaro adder (Sec. IV, Sec. VI) ------

@pytest.mark.parametrize("nb", [1, 2, 3])
def test_extended_reading_keeps_the_state(nb):
    """Extended COALESCE (ROTATE to computational-basis form, COALESCE, ROTATE
    back) on the adder with superposed inputs: the same state as the state
    vector, and every frame's matrix made of Z_k-rows after the canonical
    circuit of its own tableau."""
    ops = c.cuccaro(nb, superpose=True, toffoli="cofactor", coalesce=False)
    n = 2 * nb + 2
    mf = mfo.MultiFrameOracle(n, reading="extended")
    dense = oracle.DenseOracle(n)
    c.run(mf, ops)
    c.run(dense, ops)
    dense_equal(mf, dense, n)
    for F in mf.frames:
        x, z, _ = F.tableau()
        G = oracle.FrameOracle(n)
        sig, amp = F.frame()
        G.set_state(x, z, sig, amp)
        G.apply_clifford(mfo.canonical_circuit(x, z, n))
        gx, gz, _ = G.tableau()
        assert len(mfo.zk_rows(gx, gz)) == n


def test_state_counts_of_both_readings():
    """States at the end of the adder, nb = 1..5: the printed reading grows
    about 2.45x per bit, the extended one exactly 2x; neither is linear."""
    want = {"printed": [2, 4, 10, 22, 54], "extended": [2, 4, 8, 16, 32]}
    for reading, counts in want.items():
        got = []
        for nb in range(1, 6):
            mf = mfo.MultiFrameOracle(2 * nb + 2, reading=reading)
            c.run(mf, c.cuccaro(nb, superpose=True, toffoli="cofactor", coalesce=False))
            got.append(mf.count()[1])
        assert got == counts, (reading, got)


def _affine(points):
    t0 = next(iter(points))
    return all((a ^ b ^ t0) in points for a in points for b in points) and \
        len(points) & (len(points) - 1) == 0


@pytest.mark.parametrize("nb", [2, 3])
def test_middle_of_the_adder_has_no_coalescable_pair(nb):
    """After the MAJ chain the state is a sum over the propagate pattern p of
    2^nb stabilizer states with disjoint supports, each the graph of a linear
    map that differs for every p; no two of them sum to a stabilizer state (the
    union of their supports is never an affine space), so pairwise COALESCE
    cannot go below 2^nb states there.  The extended reading reaches exactly
    that decomposition."""
    n = 2 * nb + 2
    ops = c.cuccaro(nb, superpose=True, toffoli="cofactor", coalesce=False)[:2 * nb + 3 * nb]
    assert sum(op[0] == "T3" for op in ops) == nb
    mf = mfo.MultiFrameOracle(n, reading="extended")
    c.run(mf, ops)
    assert mf.count() == (1 << nb, 1 << nb)
    supports = []
    for F in mf.frames:
        supports.append({y for y in range(1 << n) if abs(F.amplitude(y)) > 1e-9})
    assert all(_affine(s) for s in supports)
    for i in range(len(supports)):
        for k in range(i + 1, len(supports)):
            assert not (supports[i] & supports[k])
            assert not _affine(supports[i] | supports[k])
