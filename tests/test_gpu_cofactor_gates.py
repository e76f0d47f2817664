"""Toffoli and controlled-R(alpha) by cofactors (Eq. 2, Eq. 3) on the GPU
against the oracle's implementation of the same steps: tableau and phase
vectors bit for bit, amplitudes within 1e-10, after every kind of circuit
around them (Clifford, T, measurements), across word-boundary qubit counts;
the Cuccaro adder with direct Toffolis."""
import numpy as np
import pytest

import oracle
from oracle.dense import DenseOracle
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


def circuit(n, seed, length=120):
    g = c.rng_for(seed)
    ops = []
    for op in c.random_clifford(n, length, seed=seed, kinds=(c.H, c.S, c.CNOT, c.CZ)):
        ops.append(op)
        r = g.random()
        if r < 0.05:
            a, b, t = (int(x) for x in g.choice(n, size=3, replace=False))
            ops.append(("T3", a, b, t))
        elif r < 0.08:
            a, b = (int(x) for x in g.choice(n, size=2, replace=False))
            ops.append(("CR", a, b, float(g.uniform(-3, 3))))
        elif r < 0.10:
            ops += [("N", c.T, int(g.integers(n)), 0, 0.0), ("K",)]
        elif r < 0.11:
            ops.append(("M", int(g.integers(n)), float(g.random())))
    return ops


@pytest.mark.parametrize("n,seed", [(3, 0), (5, 1), (12, 2), (40, 3), (63, 4), (64, 5), (70, 6), (130, 7)])
def test_cofactor_gates_match_oracle(sfm, n, seed):
    ops = circuit(n, 31 * n + seed)
    assert any(op[0] == "T3" for op in ops) and any(op[0] == "CR" for op in ops)
    f = sfm.Frame(n, 1 << 14)
    o = oracle.FrameOracle(n)
    rg = c.run(f, ops)
    ro = c.run(o, ops)
    assert [r[3] for r in rg] == [r[3] for r in ro]
    frames_equal(f, o)
    f.close()


def test_toffoli_state_equals_dense(sfm):
    """The frame expands to the dense state with the Toffoli applied."""
    n = 6
    ops = c.random_clifford_t(n, 60, 3, 9, t_kinds=(c.T, c.TDG)) + [("T3", 0, 3, 5), ("T3", 5, 1, 2)]
    f, d = sfm.Frame(n, 256), DenseOracle(n)
    c.run(f, ops)
    c.run(d, ops)
    got = np.array([f.amplitude(y) for y in range(1 << n)])
    assert np.max(np.abs(got - d.state())) <= TOL
    f.close()


@pytest.mark.parametrize("nb", [2, 3, 5])
def test_cuccaro_direct_toffoli(sfm, nb):
    """The adder with direct Toffolis: the oracle's frame on the equal
    superposition, and a + b on basis inputs."""
    n = 2 * nb + 2
    ops = c.cuccaro(nb, True, toffoli="cofactor")
    f, o = sfm.Frame(n, 1 << 16), oracle.FrameOracle(n)
    c.run(f, ops)
    c.run(o, ops)
    frames_equal(f, o)
    f.close()
    g = c.rng_for(nb)
    for _ in range(3):
        av, bv = int(g.integers(1 << nb)), int(g.integers(1 << nb))
        f = sfm.Frame(n, 64)
        c.run(f, c.cuccaro(nb, False, av, bv, toffoli="cofactor"))
        assert f.size() == 1 and abs(f.amplitude(c.cuccaro_reference(nb, av, bv)) - 1) <= TOL
        f.close()


def test_bad_qubits(sfm):
    f = sfm.Frame(4, 16)
    for args in ((0, 0, 1), (0, 1, 1), (0, 1, 4)):
        with pytest.raises(sfm.SFError):
            f.apply_toffoli_cofactor(*args)
    with pytest.raises(sfm.SFError):
        f.apply_cr_cofactor(2, 2, 0.5)
    f.close()
