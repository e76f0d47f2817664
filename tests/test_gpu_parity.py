"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tableau and phase vectors must match bit for bit; amplitudes and
probabilities within 1e-10 (the benchmark spec's tolerance), with the global phase
included."""
import math

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
    assert gr == orr, (gr, orr)
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz), "tableau differs"
    gs, ga = g.frame()
    os_, oa = o.frame()
    assert gs.shape == os_.shape, (gs.shape, os_.shape)
    assert np.array_equal(gs, os_), "phase vectors differ"
    if len(ga):
        err = np.max(np.abs(ga - oa))
        assert err <= tol, err
    return len(gs)


def run_both(sfm, n, ops, cap=1 << 16):
    g = sfm.Frame(n, cap)
    o = oracle.FrameOracle(n)
    rg = c.run(g, ops)
    ro = c.run(o, ops)
    for a, b in zip(rg, ro):
        assert abs(a[1] - b[1]) <= TOL and abs(a[2] - b[2]) <= TOL and a[3] == b[3]
    return g, o


def test_initial_state(sfm):
    for n in (1, 5, 64, 65, 130):
        g = sfm.Frame(n, 64)
        x, z, r = g.tableau()
        assert r == 0 and not x.any()
        for h in range(n):
            assert int(z[h, h // 64]) == 1 << (h % 64)
        s, a = g.frame()
        assert len(s) == 1 and not s.any() and abs(a[0] - 1) < 1e-15


@pytest.mark.parametrize("seed", range(100))
def test_random_clifford_t_n8(sfm, seed):
    """200 gates on 8 qubits, exactly 4 T at random positions (frame <= 16)."""
    ops = c.random_clifford_t(8, 200, 4, seed)
    g, o = run_both(sfm, 8, ops)
    k = frames_equal(g, o)
    assert k <= 16


@pytest.mark.parametrize("seed", range(4))
def test_random_clifford_t_n8_amplitudes_vs_dense(sfm, seed):
    ops = c.random_clifford_t(8, 200, 4, seed, t_kinds=(c.T, c.TDG))
    g = sfm.Frame(8, 256)
    d = DenseOracle(8)
    c.run(g, ops)
    c.run(d, ops)
    amps = np.array([g.amplitude(y) for y in range(256)])
    assert np.max(np.abs(amps - d.state())) <= TOL


@pytest.mark.parametrize("n,seed", [(3, 0), (6, 1), (7, 2), (12, 3), (33, 4), (64, 5), (65, 6), (100, 7),
                                    (127, 8), (128, 9), (129, 10), (256, 11), (257, 12), (513, 13),
                                    (1000, 14), (1024, 15)])
def test_all_kinds_mixed(sfm, n, seed):
    """All nine Clifford kinds, single and batched, with T, T-dagger, phase and
    controlled-phase gates interleaved; n spans one and several words."""
    g0 = c.rng_for(1000 + seed)
    ops = []
    for blk in range(6):
        ops += c.random_clifford(n, 25, seed * 10 + blk, kinds=tuple(range(9)))
        q = int(g0.integers(n))
        q2 = (q + 1 + int(g0.integers(n - 1))) % n if n > 1 else q
        kind = int(g0.integers(4)) if n > 1 else int(g0.integers(3))
        ops.append(("N", kind, q, q2, float(g0.random() * 2 * math.pi)))
        ops.append(("K",))
    g, o = run_both(sfm, n, ops, cap=1 << 12)
    frames_equal(g, o)


@pytest.mark.parametrize("n,seed", [(64, 0), (300, 1), (1024, 2)])
def test_long_monomial_runs(sfm, n, seed):
    """Runs of monomial gates (every kind but H) on a scrambled tableau: one
    longer than the tableau kernel holds back before a repair, one that
    changes more columns than it lists, short ones; each ended by H gates
    whose paired basis point the run's CNOTs and SWAPs have moved; T gates and
    coalescing between the blocks."""
    g0 = c.rng_for(3000 + seed)
    mono = tuple(k for k in range(9) if k != c.H)
    ops = c.random_clifford(n, min(3 * n, 600), seed + 77)
    for blk, length in enumerate((700, 60, 5, 1)):
        ops += c.random_clifford(n, length, seed * 10 + blk, kinds=mono)
        for _ in range(3):
            ops.append(("C", c.H, int(g0.integers(n)), 0))
        ops += [("N", c.T, int(g0.integers(n)), 0, 0.0), ("K",)]
    g, o = run_both(sfm, n, ops, cap=1 << 10)
    frames_equal(g, o)


def test_batched_vs_single_clifford(sfm):
    n = 10
    ops = c.random_clifford_t(n, 300, 5, 17, t_kinds=(c.T, c.TDG))
    g1 = sfm.Frame(n, 1024)
    g2 = sfm.Frame(n, 1024)
    c.run(g1, ops, batch_cliffords=True)
    c.run(g2, ops, batch_cliffords=False)
    s1, a1 = g1.frame()
    s2, a2 = g2.frame()
    assert np.array_equal(s1, s2) and np.max(np.abs(a1 - a2)) <= TOL


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_qft_parity(sfm, n):
    x, ops = c.qft_random_input(n, n)
    g, o = run_both(sfm, n, ops, cap=1 << (n + 2))
    frames_equal(g, o)
    for y in range(0, 1 << n, max(1, (1 << n) // 64)):
        assert abs(g.amplitude(y) - c.qft_expected_amplitude(n, x, y)) <= TOL


def test_qft_n16_full_frame(sfm):
    x, ops = c.qft_random_input(16, 3)
    g, o = run_both(sfm, 16, ops, cap=1 << 18)
    k = frames_equal(g, o)
    L = x.bit_length()
    assert k == (1 << (L - 1) if L else 1)


@pytest.mark.parametrize("seed", [0, 1])
def test_qft_n20_full_size(sfm, seed):
    """The QFT workload at n = 20: frame size 2^{L-1}, unit norm, sampled
    amplitudes against the closed form."""
    n = 20
    x, ops = c.qft_random_input(n, seed)
    g = sfm.Frame(n, 1 << 21)
    c.run(g, ops)
    s, a = g.frame()
    L = x.bit_length()
    assert len(s) == (1 << (L - 1) if L else 1)
    assert abs(np.sum(np.abs(a) ** 2) - 1) <= TOL
    rng = c.rng_for(seed + 7)
    for y in rng.integers(0, 1 << n, size=24):
        assert abs(g.amplitude(int(y)) - c.qft_expected_amplitude(n, x, int(y))) <= TOL


@pytest.mark.parametrize("nb", [2, 3])
def test_cuccaro_superposition_parity(sfm, nb):
    ops = c.cuccaro(nb, True)
    g, o = run_both(sfm, 2 * nb + 2, ops, cap=1 << 12)
    frames_equal(g, o)


def test_cuccaro_basis_inputs(sfm):
    nb = 4
    rng = c.rng_for(5)
    for _ in range(12):
        av, bv = int(rng.integers(16)), int(rng.integers(16))
        g = sfm.Frame(2 * nb + 2, 1 << 12)
        c.run(g, c.cuccaro(nb, False, av, bv))
        assert g.size() == 1
        assert abs(g.amplitude(c.cuccaro_reference(nb, av, bv)) - 1) <= TOL


def test_cuccaro_7bit_sampling(sfm):
    """16 qubits, peak frame 2^16: sampled outputs satisfy s = a + b, ancilla 0,
    and each sampled basis state has |amplitude| = 2^-7."""
    nb = 7
    nq = 2 * nb + 2
    anc, a, b, z = c.cuccaro_layout(nb)
    ops = c.cuccaro(nb, True)
    g = sfm.Frame(nq, 1 << 18)
    c.run(g, ops)
    for seed in range(2):
        g2 = sfm.Frame(nq, 1 << 18)
        c.run(g2, ops)
        res = c.run(g2, c.cuccaro_sample_ops(nb, seed))
        out = sum(r[3] << r[0] for r in res)
        av = sum(((out >> a[i]) & 1) << i for i in range(nb))
        sv = sum(((out >> b[i]) & 1) << i for i in range(nb)) + (((out >> z) & 1) << nb)
        assert (out >> anc) & 1 == 0
        bv = sv - av
        assert 0 <= bv < (1 << nb)
        assert abs(abs(g.amplitude(out)) - 2 ** (-nb)) <= TOL


@pytest.mark.parametrize("seed", range(10))
def test_measurement_parity(sfm, seed):
    n = 8
    ops = c.random_clifford_t(n, 120, 4, seed) + c.cuccaro_sample_ops(3, seed)[:n]
    g, o = run_both(sfm, n, ops, cap=1 << 10)
    frames_equal(g, o)


@pytest.mark.parametrize("n,seed", [(64, 0), (130, 1), (300, 2), (1024, 3)])
def test_measurement_wide(sfm, n, seed):
    """Random and deterministic measurements with collapse on multi-word
    tableaux up to the largest n, interleaved with Clifford and T gates."""
    g0 = c.rng_for(2000 + seed)
    ops = []
    for blk in range(5):
        ops += c.random_clifford(n, 30, seed * 10 + blk, kinds=(c.H, c.S, c.CNOT, c.CZ, c.SWAP))
        q = int(g0.integers(n))
        ops += [("C", c.H, q, 0), ("N", c.T, q, 0, 0.0), ("K",)]
        for _ in range(2):
            ops.append(("M", int(g0.integers(n)), float(g0.random())))
    g, o = run_both(sfm, n, ops, cap=1 << 10)
    frames_equal(g, o)


def test_probabilities_without_collapse(sfm):
    n = 7
    ops = c.random_clifford_t(n, 90, 4, 3) + [("M", q, None) for q in range(n)]
    g, o = run_both(sfm, n, ops, cap=1 << 10)
    frames_equal(g, o)


def test_device_gate_list(sfm):
    import torch
    n = 9
    ops = c.random_clifford(n, 150, 4, kinds=tuple(range(9)))
    gates = np.array([[op[1], op[2], op[3], 0] for op in ops], dtype=np.uint32)
    dev = torch.from_numpy(gates.view(np.int32)).cuda()
    g = sfm.Frame(n, 64)
    g.apply_clifford_device(dev.data_ptr(), len(gates))
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(g, o)


def test_capacity_error_is_reported_and_state_kept(sfm):
    n = 6
    g = sfm.Frame(n, 4)
    g.apply_clifford([(c.H, q, 0) for q in range(n)])
    g.apply_nonclifford(c.T, 0)
    g.coalesce()
    g.apply_nonclifford(c.T, 1)
    g.coalesce()
    assert g.size() == 4
    g.apply_nonclifford(c.T, 2)      # would need 8 children
    with pytest.raises(sfm.SFError) as ei:
        g.sync()
    assert ei.value.code == sfm.SF_ECAPACITY
    o = oracle.FrameOracle(n)
    c.run(o, [("C", c.H, q, 0) for q in range(n)] + [("N", c.T, 0, 0, 0.0), ("K",), ("N", c.T, 1, 0, 0.0), ("K",)])
    frames_equal(g, o)
    g.reset()
    g.sync()
    assert g.size() == 1


def test_invalid_arguments(sfm):
    g = sfm.Frame(4, 16)
    for bad in [lambda: g.apply_clifford([(c.H, 4, 0)]), lambda: g.apply_clifford([(c.CNOT, 1, 1)]),
                lambda: g.apply_clifford([(9, 0, 0)]), lambda: g.apply_nonclifford(c.T, 7),
                lambda: g.apply_nonclifford(c.CPHASE, 2, 2, 0.3), lambda: g.measure(5),
                lambda: g.measure(0, 2)]:
        with pytest.raises(sfm.SFError) as ei:
            bad()
        assert ei.value.code == sfm.SF_EINVAL
    g.sync()


def test_collapse_on_zero_probability(sfm):
    g = sfm.Frame(2, 16)
    p0, p1 = g.measure(0)
    assert p0 == pytest.approx(1.0) and p1 == 0.0
    with pytest.raises(sfm.SFError) as ei:
        g.measure(0, 1)
    assert ei.value.code == sfm.SF_ESTATE


def test_exact_cancellation_drops_elements(sfm):
    """T then T-dagger on a superposed qubit returns to one element."""
    g = sfm.Frame(3, 64)
    g.apply_clifford([(c.H, 0, 0), (c.CNOT, 0, 1)])
    g.apply_nonclifford(c.T, 0)
    assert g.coalesce(sync=True) == 2
    g.apply_nonclifford(c.TDG, 0)
    assert g.coalesce(sync=True) == 1
    s, a = g.frame()
    assert abs(a[0] - 1) <= TOL


def test_empty_gate_batch_is_a_no_op(sfm):
    g = sfm.Frame(5, 16)
    g.apply_clifford([])
    g.coalesce()
    assert g.size() == 1


class _Unfused:
    """The same frame driven with separate branch and coalesce calls."""

    def __init__(self, g):
        self.g = g

    def __getattr__(self, name):
        if name == "apply_nonclifford_coalesce":
            raise AttributeError(name)
        return getattr(self.g, name)


@pytest.mark.parametrize("seed", range(6))
def test_fused_and_separate_merge_agree(sfm, seed):
    n = 9 if seed % 2 else 70
    ops = c.random_clifford_t(n, 150, 5, seed, t_kinds=(c.T, c.TDG)) + [("N", c.CPHASE, 0, 1, 0.37), ("K",)]
    g1 = sfm.Frame(n, 1 << 10)
    g2 = sfm.Frame(n, 1 << 10)
    c.run(g1, ops)
    c.run(_Unfused(g2), ops)
    o = oracle.FrameOracle(n)
    c.run(o, ops)
    frames_equal(g1, o)
    frames_equal(g2, o)


def test_graph_replay_matches_eager(sfm):
    """A step captured in a CUDA graph (device gate lists, fused merges) and
    replayed several times, with the host bookkeeping restored after each
    replay, gives the eager result every time (measurement tail included)."""
    import torch
    n = 14
    x, ops = c.qft_random_input(n, 4)
    cl = [op for op in ops if op[0] == "C"]
    stream = torch.cuda.Stream()
    g = sfm.Frame(n, 1 << (n + 2), stream=stream)
    seq = []
    pending = []
    for op in ops:
        if op[0] == "C":
            pending.append(op)
            continue
        if pending:
            arr = np.array([[p[1], p[2], p[3], 0] for p in pending], dtype=np.uint32)
            seq.append(("C", torch.from_numpy(arr.view(np.int32)).cuda()))
            pending = []
        seq.append(op)

    def async_part():
        g.reset()
        for op in seq:
            if op[0] == "C":
                g.apply_clifford_device(op[1].data_ptr(), op[1].shape[0])
            elif op[0] == "N":
                g.apply_nonclifford_coalesce(op[1], op[2], op[3], op[4], 1e-12)

    with torch.cuda.stream(stream):
        async_part()
    p_ref = g.measure(0)
    s_ref, a_ref = g.frame()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        async_part()
    token = g.host_state()
    for _ in range(3):
        with torch.cuda.stream(stream):
            graph.replay()
        g.set_host_state(token)
        p = g.measure(0)
        s, a = g.frame()
        assert abs(p[0] - p_ref[0]) <= TOL
        assert np.array_equal(s, s_ref) and np.max(np.abs(a - a_ref)) <= TOL
