"""Exhaustive small cases of the frame oracle against the state vector.

Every n-qubit stabilizer state for n = 1, 2, 3 is reached from |0...0> by H, S
and CNOT (breadth-first, states equal up to a global phase counted once); their
number must be 2^n prod_{k=1..n} (2^k + 1) = 6, 60, 1080, the count of
stabilizer states (Aaronson & Gottesman), which pins the enumeration itself.
From each state the frame oracle -- which reaches it by the same gates and
tracks its global phase -- must equal the state vector after every Clifford
kind on every qubit choice, after T on every qubit, and in its measurement
probabilities and amplitudes (Sec. II-B, Table 2, Sec. III, Sec. IV)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import DenseOracle
from paper_1712_03554_gb300 import circuits as c

TOL = 1e-12


def stabilizer_state_count(n):
    return 2 ** n * int(np.prod([2 ** k + 1 for k in range(1, n + 1)]))


def phase_free_key(v):
    j = int(np.flatnonzero(np.abs(v) > 1e-9)[0])
    w = v * (abs(v[j]) / v[j])
    return tuple(np.round(w.real, 9)) + tuple(np.round(w.imag, 9))


def orbit(n):
    """[(gate path, dense vector)] for every stabilizer state of n qubits."""
    gens = [(c.H, q, 0) for q in range(n)] + [(c.S, q, 0) for q in range(n)]
    gens += [(c.CNOT, a, b) for a, b in itertools.permutations(range(n), 2)]
    d = DenseOracle(n)
    seen = {phase_free_key(d.state()): ([], d.state())}
    frontier = [([], d.state())]
    while frontier:
        nxt = []
        for path, v in frontier:
            for g in gens:
                d.psi = v.copy()
                d.apply_clifford([g])
                key = phase_free_key(d.psi)
                if key not in seen:
                    seen[key] = (path + [g], d.state())
                    nxt.append(seen[key])
        frontier = nxt
    return list(seen.values())


ORBITS = {n: orbit(n) for n in (1, 2, 3)}


def gate_set(n):
    gates = [(k, q, 0) for k in (c.H, c.S, c.SDG, c.X, c.Y, c.Z) for q in range(n)]
    gates += [(k, a, b) for k in (c.CNOT, c.CZ, c.SWAP) for a, b in itertools.permutations(range(n), 2)]
    return gates


def frame_vector(f, n):
    return np.array([f.amplitude(y) for y in range(1 << n)])


@pytest.mark.parametrize("n", [1, 2, 3])
def test_orbit_is_every_stabilizer_state(n):
    assert len(ORBITS[n]) == stabilizer_state_count(n)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_every_state_every_clifford(n):
    """Each stabilizer state (each M and each sigma) under each Clifford kind
    on each qubit choice, global phase included."""
    gates = gate_set(n)
    for path, v in ORBITS[n]:
        f0 = oracle.FrameOracle(n)
        if path:
            f0.apply_clifford(path)
        assert np.allclose(frame_vector(f0, n), v, atol=TOL)
        x, z, _ = f0.tableau()
        sig, amp = f0.frame()
        for g in gates:
            f = oracle.FrameOracle(n)
            f.set_state(x, z, sig, amp)
            f.apply_clifford([g])
            d = DenseOracle(n)
            d.psi = v.copy()
            d.apply_clifford([g])
            assert f.is_rref()
            assert np.allclose(frame_vector(f, n), d.state(), atol=TOL), (path, g)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_every_state_t_branch_measure_amplitude(n):
    """T on every qubit (branching by the anticommutation mask and Def. 1
    coalescing), the measurement probabilities of every qubit (COFACTOR when
    the outcome is random) and Observation 1's amplitudes."""
    for path, v in ORBITS[n]:
        f0 = oracle.FrameOracle(n)
        if path:
            f0.apply_clifford(path)
        x, z, _ = f0.tableau()
        sig, amp = f0.frame()
        for q in range(n):
            f = oracle.FrameOracle(n)
            f.set_state(x, z, sig, amp)
            f.apply_nonclifford(c.T, q)
            f.coalesce()
            d = DenseOracle(n)
            d.psi = v.copy()
            d.apply_nonclifford(c.T, q)
            assert np.allclose(frame_vector(f, n), d.state(), atol=TOL), (path, q)
            assert f.size() <= 2
            g = oracle.FrameOracle(n)
            g.set_state(x, z, sig, amp)
            p = g.measure(q, -1)
            d.psi = v.copy()
            assert np.allclose(p, d.measure(q, -1), atol=TOL), (path, q)
