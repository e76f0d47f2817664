"""Multiframe simulation on the GPU (include/sf_multiframe.h, Sec. IV) against
the multiframe oracle: the same frames (stabilizer matrices and phase vectors
bit for bit), amplitudes within 1e-10, the same counts, and the state-vector
oracle's amplitudes; capacity and argument errors."""
import math

import pytest

import oracle
from oracle import multiframe as mfo
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


def same_multiframe(g, o):
    gd, od = g.as_dict(), o.as_dict()
    assert set(gd) == set(od), "stabilizer matrices differ"
    for key, elems in od.items():
        assert set(gd[key]) == set(elems), "phase vectors differ"
        for s, a in elems.items():
            assert abs(gd[key][s] - a) <= TOL
    assert g.count() == o.count()


def test_paper_example(sfm):
    g = sfm.MultiFrame(3, 64, 16)
    o = mfo.MultiFrameOracle(3)
    for sim in (g, o):
        sim.apply_clifford([(c.H, 0, 0), (c.H, 1, 0)])
        sim.apply_toffoli_cofactor(0, 1, 2)
    assert g.count() == (2, 2)
    same_multiframe(g, o)
    assert g.kernel_launches() > 0
    g.close()


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5])
def test_cuccaro_superposition(sfm, nb):
    ops = c.cuccaro(nb, superpose=True, toffoli="cofactor", coalesce=False)
    n = 2 * nb + 2
    g = sfm.MultiFrame(n, 4096, 4096)
    o = mfo.MultiFrameOracle(n)
    c.run(g, ops)
    c.run(o, ops)
    same_multiframe(g, o)
    for y in c.rng_for(nb).integers(1 << n, size=6):
        assert abs(g.amplitude(int(y)) - o.amplitude(int(y))) <= TOL
    g.close()


@pytest.mark.parametrize("nb,a,b", [(4, 9, 11), (6, 45, 27)])
def test_cuccaro_basis_inputs(sfm, nb, a, b):
    ops = c.cuccaro(nb, superpose=False, a_val=a, b_val=b, toffoli="cofactor", coalesce=False)
    g = sfm.MultiFrame(2 * nb + 2, 256, 64)
    c.run(g, ops)
    assert g.count() == (1, 1)
    assert abs(g.amplitude(c.cuccaro_reference(nb, a, b)) - 1.0) <= TOL
    g.close()


@pytest.mark.parametrize("seed", range(8))
def test_random_circuits(sfm, seed):
    """Clifford gates, Toffolis and controlled-R(alpha) with alpha in
    {pi, +-pi/2, pi/4} (pairs with d = 0, 1, 2, 3), T gates branched inside the
    frames; the multiframe is compared after every non-Clifford gate."""
    g_ = c.rng_for(4200 + seed)
    n = int(g_.integers(4, 11))
    g = sfm.MultiFrame(n, 4096, 4096)
    o = mfo.MultiFrameOracle(n)
    dense = oracle.DenseOracle(n)
    for step in range(12):
        gates = []
        for _ in range(int(g_.integers(1, 5))):
            kind = int(g_.choice([c.H, c.S, c.CNOT, c.X, c.CZ]))
            q0 = int(g_.integers(n))
            q1 = int((q0 + 1 + g_.integers(n - 1)) % n) if kind in (c.CNOT, c.CZ) else 0
            gates.append((kind, q0, q1))
        for sim in (g, o, dense):
            sim.apply_clifford(gates)
        a, b, t = (int(v) for v in g_.choice(n, size=3, replace=False))
        r = step % 4
        if r == 3:
            alpha = float(g_.choice([math.pi, math.pi / 2, -math.pi / 2, math.pi / 4]))
            for sim in (g, o, dense):
                sim.apply_cr_cofactor(a, t, alpha)
        elif r == 2 and step < 8:
            g.apply_nonclifford_coalesce(c.T, a)
            o.apply_nonclifford_coalesce(c.T, a)
            dense.apply_nonclifford(c.T, a)
        else:
            for sim in (g, o, dense):
                sim.apply_toffoli_cofactor(a, b, t)
        same_multiframe(g, o)
    for y in range(min(1 << n, 64)):
        assert abs(g.amplitude(y) - dense.amplitude(y)) <= TOL
    g.close()


def phase_product(sim, n):
    """H on every qubit, P(+-pi/2) branched on each (one frame of 2^n
    elements whose amplitude ratios are powers of i), H on every qubit again:
    every row becomes a Z_k-row."""
    sim.apply_clifford([(c.H, q, 0) for q in range(n)])
    for q in range(n):
        sim.apply_nonclifford_coalesce(c.PHASE, q, 0, math.pi / 2 if q % 3 else -math.pi / 2)
    sim.apply_clifford([(c.H, q, 0) for q in range(n)])


@pytest.mark.parametrize("n", [12, 13])
def test_large_frame(sfm, n):
    """COALESCE of one frame of 4096 / 8192 elements (the largest one CTA
    sorts): the multiframe collapses to the product state's single element."""
    g = sfm.MultiFrame(n, 1 << n, 64)
    o = mfo.MultiFrameOracle(n)
    for sim in (g, o):
        phase_product(sim, n)
    assert g.count() == o.count() == (1, 1 << n)
    assert g.coalesce() == o.coalesce() == (1, 1)
    same_multiframe(g, o)
    g.close()


def test_errors(sfm):
    with pytest.raises(sfm.SFError) as e:
        sfm.MultiFrame(64, 16, 4)
    assert e.value.code == sfm.SF_EINVAL
    # two frames needed, one allowed
    g = sfm.MultiFrame(3, 64, 1)
    g.apply_clifford([(c.H, 0, 0), (c.H, 1, 0)])
    with pytest.raises(sfm.SFError) as e:
        g.apply_toffoli_cofactor(0, 1, 2)
    assert e.value.code == sfm.SF_ECAPACITY
    g.close()
    # bad Toffoli qubits are rejected and the multiframe stays usable
    g = sfm.MultiFrame(4, 64, 8)
    with pytest.raises(sfm.SFError) as e:
        g.apply_toffoli_cofactor(0, 0, 2)
    assert e.value.code == sfm.SF_EINVAL
    g.apply_clifford([(c.H, 0, 0)])
    g.apply_toffoli_cofactor(0, 1, 2)
    assert g.count() == (1, 1)  # the two cofactors of qubit 0 pair again
    with pytest.raises(sfm.SFError):
        g.frame(5)
    g.close()
    # a frame above the largest COALESCE sorts
    g = sfm.MultiFrame(14, 1 << 14, 8)
    phase_product(g, 14)
    with pytest.raises(sfm.SFError) as e:
        g.coalesce()
    assert e.value.code == sfm.SF_ECAPACITY
    g.close()
