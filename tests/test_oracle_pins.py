"""Pins of the CPU oracle to facts outside itself (tables, worked examples of the
paper, closed forms, brute force).  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle.dense import (DenseOracle, ONE_QUBIT, PAULI, pauli_row_matrix,
                          stabilizer_state_by_projection, two_qubit_matrix)
from paper_1712_03554_gb300 import circuits as c

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LIT = {"I": 0, "Z": 1, "X": 2, "Y": 3}
PH = {"1": 0, "i": 1, "-1": 2, "-i": 3}


def _rows(path):
    with open(path) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


# ---- Table 1 -------------------------------------------------------------------
def test_table1_pauli_products():
    rows = _rows(os.path.join(GOLDEN, "table1_pauli_products.txt"))
    assert len(rows) == 16
    for a, b, ph, res in rows:
        k, lit = oracle.pauli_mult(LIT[a], LIT[b])
        assert (k, lit) == (PH[ph], LIT[res]), (a, b)
        # the table itself agrees with the 2x2 matrices
        assert np.allclose(PAULI[LIT[a]] @ PAULI[LIT[b]], (1j ** PH[ph]) * PAULI[LIT[res]])


# ---- Table 2 -------------------------------------------------------------------
def test_table2_conjugation_rows():
    kinds = {"H": c.H, "P": c.S, "CNOT": c.CNOT}
    for gate, inp, out, sgn in _rows(os.path.join(GOLDEN, "table2_conjugation.txt")):
        l0, l1 = LIT[inp[0]], (LIT[inp[1]] if len(inp) > 1 else 0)
        s, o0, o1 = oracle.conjugate(kinds[gate], l0, l1)
        want0, want1 = LIT[out[0]], (LIT[out[1]] if len(out) > 1 else 0)
        assert (s, o0, o1) == (1 if sgn == "-" else 0, want0, want1), (gate, inp)


def _dense_gate(kind):
    if kind in ONE_QUBIT:
        return ONE_QUBIT[kind], 1
    return two_qubit_matrix(kind), 2


def test_dense_gate_matrices_are_the_textbook_ones():
    H, S, X, Z = ONE_QUBIT[0], ONE_QUBIT[1], ONE_QUBIT[3], ONE_QUBIT[5]
    assert np.allclose(H, (X + Z) / math.sqrt(2))
    assert np.allclose(S @ S, Z) and np.allclose(ONE_QUBIT[2], S.conj().T)
    assert np.allclose(ONE_QUBIT[4], 1j * X @ Z)
    cn = two_qubit_matrix(c.CNOT)   # local index bit0 = control, bit1 = target
    assert cn[3, 1] == 1 and cn[1, 3] == 1 and cn[0, 0] == 1 and cn[2, 2] == 1
    assert np.allclose(two_qubit_matrix(c.CZ), np.diag([1, 1, 1, -1]))


@pytest.mark.parametrize("kind", list(range(9)))
def test_conjugation_all_kinds_exhaustive(kind):
    """Every literal (pair) conjugated by every Clifford kind matches U P U^dagger."""
    U, nq = _dense_gate(kind)
    for lits in itertools.product(range(4), repeat=nq):
        l0, l1 = lits[0], (lits[1] if nq == 2 else 0)
        s, o0, o1 = oracle.conjugate(kind, l0, l1)
        if nq == 1:
            P, Q = PAULI[l0], PAULI[o0]
        else:  # local index bit0 = q0 -> q0 is the least significant factor
            P, Q = np.kron(PAULI[l1], PAULI[l0]), np.kron(PAULI[o1], PAULI[o0])
        assert np.allclose(U @ P @ U.conj().T, (-1) ** s * Q), (kind, lits)


# ---- worked examples -------------------------------------------------------------
def test_example1_bell_matrices():
    """Ex. 1: (|00>+|11>)/sqrt2 has M1 = [+XX,+ZZ]; M2 = [+XX,-YY] and M3 = [-YY,+ZZ]
    follow by row products; the canonical form is +XX, +ZZ with one element a=1."""
    f = oracle.FrameOracle(2)
    f.apply_clifford([(c.H, 0, 0), (c.CNOT, 0, 1)])
    x, z, r = f.tableau()
    assert r == 1 and list(x[:, 0]) == [3, 0] and list(z[:, 0]) == [0, 3]
    sig, amp = f.frame()
    assert list(sig[:, 0]) == [0] and np.allclose(amp, [1.0])
    ph = 0
    for _ in range(2):   # XX * ZZ literal by literal
        k, res = oracle.pauli_mult(LIT["X"], LIT["Z"])
        ph += k
        assert res == LIT["Y"]
    assert ph % 4 == 2   # XX*ZZ = -YY: M2's second row


def test_example2_cnot_on_bell():
    """Ex. 2: CNOT maps [+XX, +ZZ] to [+XI, +IZ]."""
    f = oracle.FrameOracle(2)
    f.apply_clifford([(c.H, 0, 0), (c.CNOT, 0, 1), (c.CNOT, 0, 1)])
    x, z, r = f.tableau()
    assert list(x[:, 0]) == [1, 0] and list(z[:, 0]) == [0, 2] and r == 1
    sig, amp = f.frame()
    assert list(sig[:, 0]) == [0] and np.allclose(amp, [1.0])


def test_phase_gate_on_one_keeps_relative_phase():
    """Sec. II-B: P|1> = i|1> while the stabilizer stays -Z; the frame keeps the i."""
    f = oracle.FrameOracle(1)
    f.apply_clifford([(c.X, 0, 0), (c.S, 0, 0)])
    sig, amp = f.frame()
    assert list(sig[:, 0]) == [1] and np.allclose(amp, [1j])


def test_example4_two_phase_vectors():
    """Ex. 4: a1(|00>+|01>) + a2(|10>+|11>) needs two phase vectors over
    M = RREF{ZI, IX} = [IX; ZI] that differ only in the ZI sign."""
    f = oracle.FrameOracle(2)
    # qubit 0 is the paper's first qubit: a biased state on it, |+> on qubit 1
    f.apply_clifford([(c.H, 0, 0)])
    f.apply_nonclifford(c.T, 0)
    f.coalesce()
    f.apply_clifford([(c.H, 0, 0), (c.H, 1, 0)])
    x, z, r = f.tableau()
    assert r == 1 and list(x[:, 0]) == [2, 0] and list(z[:, 0]) == [0, 1]
    sig, amp = f.frame()
    assert len(sig) == 2 and int(sig[0, 0]) ^ int(sig[1, 0]) == 0b10


def test_cofactor_example_four_states():
    """Sec. III: |000>+|010>+|100>+|110> cofactored on its first two qubits
    gives four states."""
    f = oracle.FrameOracle(3)
    f.apply_clifford([(c.H, 0, 0), (c.H, 1, 0)])
    assert f.size() == 1
    f.measure(0, -1)
    f.measure(1, -1)
    sig, amp = f.frame()
    assert len(sig) == 4 and np.allclose(np.abs(amp), 0.5)
    x, z, r = f.tableau()
    assert r == 0


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz(n):
    f = oracle.FrameOracle(n)
    f.apply_clifford([(c.H, 0, 0)] + [(c.CNOT, i, i + 1) for i in range(n - 1)])
    x, z, r = f.tableau()
    assert r == 1 and int(x[0, 0]) == (1 << n) - 1 and int(z[0, 0]) == 0
    for i in range(n - 1):    # Z-block: Z_i Z_{n-1}
        assert int(x[1 + i, 0]) == 0 and int(z[1 + i, 0]) == (1 << i) | (1 << (n - 1))
    sig, amp = f.frame()
    assert list(sig[:, 0]) == [0] and np.allclose(amp, [1.0])


# ---- brute force against the dense oracle ------------------------------------------
def _expand_by_projection(f, n):
    x, z, r = f.tableau()
    sig, amp = f.frame()
    psi = np.zeros(1 << n, dtype=complex)
    for s, a in zip(sig[:, 0], amp):
        psi += a * stabilizer_state_by_projection(n, x[:, 0], z[:, 0], int(s))
    return psi


@pytest.mark.parametrize("seed", range(12))
def test_frame_expands_to_state_vector(seed):
    n = 5
    ops = c.random_clifford_t(n, 60, 3, seed, t_kinds=(c.T, c.TDG))
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    assert np.allclose(_expand_by_projection(f, n), d.state(), atol=1e-12)
    assert f.is_rref()


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_every_phase_vector(seed):
    """a_sigma = <psi_can(M, sigma)|Psi> for every sigma in {0,1}^n: the frame is
    exactly the set of sigma with |a| >= eps, with those amplitudes."""
    n = 4
    ops = c.random_clifford_t(n, 50, 3, seed) + [("N", c.CPHASE, 0, 2, 0.9), ("K",)]
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    x, z, r = f.tableau()
    sig, amp = f.frame()
    got = {int(s): a for s, a in zip(sig[:, 0], amp)}
    for s in range(1 << n):
        a = np.vdot(stabilizer_state_by_projection(n, x[:, 0], z[:, 0], s), d.state())
        if abs(a) >= 1e-12:
            assert s in got and abs(got[s] - a) < 1e-12
        else:
            assert s not in got


def test_rows_stabilize_dense_state():
    n = 6
    ops = c.random_clifford(n, 120, 3, kinds=tuple(range(9)))
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    x, z, r = f.tableau()
    sig, amp = f.frame()
    assert len(sig) == 1 and abs(abs(amp[0]) - 1) < 1e-12
    psi = d.state()
    for h in range(n):
        s = -1 if (int(sig[0, 0]) >> h) & 1 else 1
        assert np.allclose(s * pauli_row_matrix(int(x[h, 0]), int(z[h, 0]), n) @ psi, psi)


@pytest.mark.parametrize("seed", range(8))
def test_random_clifford_t_vs_dense(seed):
    n = 8
    ops = c.random_clifford_t(n, 200, 4, seed)
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    amps = np.array([f.amplitude(y) for y in range(1 << n)])
    assert np.allclose(amps, d.state(), atol=1e-12)
    sig, amp = f.frame()
    assert len(sig) <= 16 and abs(np.sum(np.abs(amp) ** 2) - 1) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_measurement_vs_dense(seed):
    n = 6
    ops = c.random_clifford_t(n, 80, 4, seed) + c.cuccaro_sample_ops(2, seed)[:n]
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    r1 = c.run(f, ops)
    r2 = c.run(d, ops)
    for a, b in zip(r1, r2):
        assert abs(a[1] - b[1]) < 1e-12 and abs(a[2] - b[2]) < 1e-12 and a[3] == b[3]
    assert np.allclose([f.amplitude(y) for y in range(1 << n)], d.state(), atol=1e-12)
    assert f.is_rref()


# ---- closed forms -------------------------------------------------------------------
@pytest.mark.parametrize("n,x", [(3, 0b111), (6, 0b101101), (9, 0x1ff), (10, 777)])
def test_qft_closed_form(n, x):
    f = oracle.FrameOracle(n)
    c.run(f, c.qft(n, x))
    for y in range(1 << n):
        assert abs(f.amplitude(y) - c.qft_expected_amplitude(n, x, y)) < 1e-12
    # frame size 2^{L-1}, L = 1-based position of the highest set bit of x
    L = x.bit_length()
    assert f.size() == (1 << (L - 1) if L else 1)


def test_toffoli_decomposition_is_toffoli():
    for a_in in range(8):
        d = DenseOracle(3)
        d.apply_clifford([(c.X, q, 0) for q in range(3) if (a_in >> q) & 1])
        c.run(d, c.toffoli_clifford_t(0, 1, 2))
        want = a_in ^ (4 if (a_in & 3) == 3 else 0)
        e = np.zeros(8, dtype=complex)
        e[want] = 1
        assert np.allclose(d.state(), e, atol=1e-12)


def test_cuccaro_classical_is_addition():
    nb = 4
    anc, a, b, z = c.cuccaro_layout(nb)
    for av in range(16):
        for bv in range(16):
            out = c.cuccaro_reference(nb, av, bv)
            s = sum(((out >> b[i]) & 1) << i for i in range(nb))
            got_a = sum(((out >> a[i]) & 1) << i for i in range(nb))
            assert got_a == av and (out >> anc) & 1 == 0
            assert s + (((out >> z) & 1) << nb) == av + bv


def test_cuccaro_frame_on_basis_inputs():
    nb = 3
    for av in range(8):
        for bv in range(8):
            f = oracle.FrameOracle(2 * nb + 2)
            c.run(f, c.cuccaro(nb, False, av, bv))
            assert f.size() == 1
            assert abs(f.amplitude(c.cuccaro_reference(nb, av, bv)) - 1) < 1e-12


def test_cuccaro_superposition_vs_dense():
    nb = 3
    ops = c.cuccaro(nb, True)
    f, d = oracle.FrameOracle(2 * nb + 2), DenseOracle(2 * nb + 2)
    c.run(f, ops)
    c.run(d, ops)
    assert np.allclose([f.amplitude(y) for y in range(1 << (2 * nb + 2))], d.state(), atol=1e-12)


def test_invariant1_after_every_op():
    n = 7
    f = oracle.FrameOracle(n)
    for op in c.random_clifford_t(n, 120, 5, 11) + c.cuccaro_sample_ops(3, 1)[:n]:
        c.run(f, [op])
        assert f.is_rref()


def test_planted_sign_error_is_caught():
    """A wrong sign in one amplitude (what a dropped i-power term would do) is
    caught by the dense expansion check."""
    n = 4
    ops = c.random_clifford_t(n, 40, 2, 3)
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    x, z, r = f.tableau()
    sig, amp = f.frame()
    amp2 = amp.copy()
    amp2[0] *= -1
    psi = np.zeros(1 << n, dtype=complex)
    for s, a in zip(sig[:, 0], amp2):
        psi += a * stabilizer_state_by_projection(n, x[:, 0], z[:, 0], int(s))
    assert not np.allclose(psi, d.state(), atol=1e-9)


# ---- Toffoli and controlled-R(alpha) by cofactors (Eq. 2, Eq. 3) -----------------
def _dense_prefix(n, seed):
    ops = c.random_clifford_t(n, 40, 3, seed, t_kinds=(c.T, c.TDG))
    f, d = oracle.FrameOracle(n), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    return f, d


@pytest.mark.parametrize("seed", range(10))
def test_cofactor_toffoli_is_the_toffoli(seed):
    """After Eq. 2 on a random Clifford+T state, the frame (expanded by
    projectors, independently of the oracle's amplitude code) is the dense
    state with the Toffoli permutation applied, global phase included; M holds
    Z_c1 and Z_c2 as rows and stays in RREF; a second Toffoli restores the
    state."""
    n = 5
    g = c.rng_for(500 + seed)
    c1, c2, t = (int(x) for x in g.choice(n, size=3, replace=False))
    f, d = _dense_prefix(n, seed)
    before = d.state()
    f.apply_toffoli_cofactor(c1, c2, t)
    d.apply_toffoli_cofactor(c1, c2, t)
    assert np.allclose(_expand_by_projection(f, n), d.state(), atol=1e-12)
    assert f.is_rref()
    x, z, r = f.tableau()
    rows = {(int(x[h, 0]), int(z[h, 0])) for h in range(n)}
    assert (0, 1 << c1) in rows and (0, 1 << c2) in rows
    f.apply_toffoli_cofactor(c1, c2, t)
    assert np.allclose(_expand_by_projection(f, n), before, atol=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_cofactor_cr_is_the_controlled_phase(seed):
    n = 5
    g = c.rng_for(700 + seed)
    ct, tt = (int(x) for x in g.choice(n, size=2, replace=False))
    alpha = float(g.uniform(-3, 3))
    f, d = _dense_prefix(n, seed)
    f.apply_cr_cofactor(ct, tt, alpha)
    d.apply_nonclifford(c.CPHASE, ct, tt, alpha)
    assert np.allclose(_expand_by_projection(f, n), d.state(), atol=1e-12)
    assert f.is_rref()


def test_cofactor_toffoli_on_basis_states_and_cuccaro():
    """Classical inputs: the Toffoli truth table with a single-element frame;
    the Cuccaro adder with direct Toffolis adds, and on the equal superposition
    equals the 7T-decomposed adder's state."""
    for a_in in range(8):
        f = oracle.FrameOracle(3)
        f.apply_clifford([(c.X, q, 0) for q in range(3) if (a_in >> q) & 1])
        f.apply_toffoli_cofactor(0, 1, 2)
        want = a_in ^ (4 if (a_in & 3) == 3 else 0)
        assert f.size() == 1 and abs(f.amplitude(want) - 1) < 1e-12
    nb = 3
    for av, bv in ((3, 5), (7, 7), (0, 6)):
        f = oracle.FrameOracle(2 * nb + 2)
        c.run(f, c.cuccaro(nb, False, av, bv, toffoli="cofactor"))
        assert abs(f.amplitude(c.cuccaro_reference(nb, av, bv)) - 1) < 1e-12
    f = oracle.FrameOracle(2 * nb + 2)
    c.run(f, c.cuccaro(nb, True, toffoli="cofactor"))
    d = DenseOracle(2 * nb + 2)
    c.run(d, c.cuccaro(nb, True))
    assert np.allclose([f.amplitude(y) for y in range(1 << (2 * nb + 2))], d.state(), atol=1e-12)
