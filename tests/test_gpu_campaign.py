"""Parity of the batched campaign engine (sf_campaign_*, one persistent launch
for many circuits) with the CPU oracle, with the one-circuit GPU path, and
with itself when a circuit runs alone instead of in a batch.

Tableau and phase vectors bit for bit; amplitudes within 1e-10 (global phase
included); measurement outcomes exactly (both sides decide u < p(1) in FP64)."""
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


def oracle_run(n, ops):
    o = oracle.FrameOracle(n)
    res = c.run(o, ops)
    bits = 0
    for m, r in enumerate(res):
        bits |= r[3] << m
    return o, bits, len(res)


def check_against_oracle(res, i, n, ops):
    o, bits, nm = oracle_run(n, ops)
    assert res["status"][i] == 0, (i, res["status"][i])
    assert int(res["outcomes"][i]) == bits, (i, bin(int(res["outcomes"][i])), bin(bits))
    assert res["n_meas"][i] == nm
    x, z, r, sig, amp = res["frames"][i]
    ox, oz, orr = o.tableau()
    assert r == orr
    assert np.array_equal(x, ox[:, 0]) and np.array_equal(z, oz[:, 0]), "tableau differs"
    os_, oa = o.frame()
    assert res["k_final"][i] == len(os_)
    assert np.array_equal(sig, os_[:, 0]), "phase vectors differ"
    if len(oa):
        assert np.max(np.abs(amp - oa)) <= TOL
    assert abs(res["norm"][i] - np.sum(np.abs(oa) ** 2)) <= TOL


def test_steane_variants_vs_oracle(sfm):
    circuits = c.steane_campaign(48, seed=1)
    eng = sfm.Campaign(c.STEANE_N, 8192)
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        check_against_oracle(res, i, c.STEANE_N, ops)
    eng.close()


@pytest.mark.parametrize("n", [1, 2, 8, 31, 32, 33, 63])
def test_random_clifford_t_vs_oracle(sfm, n):
    """All nine Clifford kinds, T/T-dagger/PHASE on one qubit and CPHASE on
    pairs, measurements with draws and conditional gates, across word-boundary
    qubit counts."""
    g = c.rng_for(1000 + n)
    circuits = []
    for v in range(6):
        ops = c.random_clifford(n, 150, seed=97 * n + v, kinds=tuple(range(9)) if n >= 2 else (0, 1, 2, 3, 4, 5))
        out = []
        n_meas = 0
        for op in ops:
            out.append(op)
            r = g.random()
            if r < 0.03:
                out += [("N", int(g.integers(3)), int(g.integers(n)), 0, float(g.uniform(-3, 3))), ("K",)]
            elif r < 0.045 and n >= 2:
                a, b = (int(x) for x in g.choice(n, size=2, replace=False))
                out += [("N", c.CPHASE, a, b, float(g.uniform(-3, 3))), ("K",)]
            elif r < 0.10:
                out.append(("M", int(g.integers(n)), float(g.random())))
                n_meas += 1
            elif r < 0.12 and n_meas:
                out.append(("Q", int(g.integers(6)), int(g.integers(n)), 0, int(g.integers(1, 1 << n_meas))))
        circuits.append(out)
    eng = sfm.Campaign(n, sfm.CAMPAIGN_MAX_ELEMS)
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        check_against_oracle(res, i, n, ops)
    eng.close()


def test_qft_vs_oracle(sfm):
    """QFT on 10 qubits from random basis states: frames grow to hundreds of
    elements through merged controlled phases."""
    circuits = []
    for s in range(4):
        x, ops = c.qft_random_input(10, seed=s)
        circuits.append(ops)
    eng = sfm.Campaign(10, 4096)
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        check_against_oracle(res, i, 10, ops)
    assert max(res["k_final"]) >= 256
    eng.close()


def test_alone_equals_batched(sfm):
    """A circuit's results do not depend on what runs beside it: bit-identical
    outputs and exported frames alone and inside a batch of 256."""
    circuits = c.steane_campaign(256, seed=2)
    eng = sfm.Campaign(c.STEANE_N, 8192)
    full = eng.run(circuits, export=True)
    for i in (0, 17, 255):
        one = eng.run([circuits[i]], export=True)
        for key in ("outcomes", "n_meas", "k_final", "norm", "status"):
            assert one[key][0] == full[key][i], key
        for a, b in zip(one["frames"][0], full["frames"][i]):
            assert np.array_equal(np.asarray(a), np.asarray(b))
    eng.close()


def test_campaign_vs_single_circuit_path(sfm):
    """The campaign and the one-circuit library path (sf_create ... per
    circuit) give the same outcomes and frames."""
    circuits = c.steane_campaign(6, seed=3)
    eng = sfm.Campaign(c.STEANE_N, 8192)
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        f = sfm.Frame(c.STEANE_N, 1 << 14)
        rr = c.run(f, ops)
        bits = sum(r[3] << m for m, r in enumerate(rr))
        assert int(res["outcomes"][i]) == bits
        gx, gz, gr = f.tableau()
        x, z, r, sig, amp = res["frames"][i]
        assert gr == r and np.array_equal(gx[:, 0], x) and np.array_equal(gz[:, 0], z)
        gs, ga = f.frame()
        assert np.array_equal(gs[:, 0], sig)
        assert np.max(np.abs(ga - amp)) <= TOL
        f.close()
    eng.close()


def test_statuses_and_edge_cases(sfm):
    """Per-circuit errors stop that circuit only; an empty circuit is |0..0>."""
    n = 6
    plus3 = [("C", c.H, q, 0) for q in range(3)] + [x for q in range(3) for x in (("N", c.T, q, 0, 0.0), ("K",))]
    circuits = [
        [],                                          # empty: one element, norm 1
        [("C", c.H, 0, 0), ("C", c.CNOT, 0, 9)],     # qubit out of range
        plus3,                                       # 8 elements > max_elems 4
        [("C", c.H, 0, 0), ("C", c.CNOT, 0, 0)],     # q0 == q1
        [("C", c.X, 0, 0), ("M", 0, 0.5), ("M", 0, 0.5)],
        [("C", c.H, 1, 0), ("N", c.T, 1, 0, 0.0), ("K",)],
    ]
    eng = sfm.Campaign(n, 4)
    res = eng.run(circuits, export=True)
    assert list(res["status"]) == [0, sfm.SF_EINVAL, sfm.SF_ECAPACITY, sfm.SF_EINVAL, 0, 0]
    assert res["k_final"][0] == 1 and abs(res["norm"][0] - 1) < 1e-15
    assert int(res["outcomes"][4]) == 0b11 and res["n_meas"][4] == 2
    assert res["k_final"][5] == 2
    # the draw decides between p(1) and p(0): u just below and above p(1) = 1/2
    h = [("C", c.H, 2, 0), ("M", 2, 0.4999999), ("C", c.H, 3, 0), ("M", 3, 0.5000001)]
    r2 = eng.run([h])
    assert int(r2["outcomes"][0]) == 0b01
    # a conditional gate must be a Clifford kind
    ops, off, nc = eng.upload([[("C", c.H, 0, 0)]])
    rec = ops.cpu().numpy().view(sfm.SF_OP_DTYPE).copy()
    rec["kind"][0], rec["arg"][0] = sfm.OP_COND, 20
    rec["param"][0] = np.array([1], dtype=np.uint64).view(np.float64)[0]
    import torch
    ops = torch.from_numpy(rec.view(np.uint8)).to("cuda")
    out = eng.outputs(1)
    eng.launch(ops, off, 1, 1e-12, out)
    torch.cuda.synchronize()
    assert int(out["status"][0]) == sfm.SF_EINVAL
    # zero circuits: nothing to do
    eng.launch(ops, off, 0, 1e-12, out)
    eng.close()
    with pytest.raises(sfm.SFError):
        sfm.Campaign(64, 16)
    with pytest.raises(sfm.SFError):
        sfm.Campaign(8, sfm.CAMPAIGN_MAX_ELEMS + 1)


def test_shapes_agree_and_autotune(sfm):
    """Every launch shape (threads per circuit x index placement) gives the
    same outcomes, frame sizes and phase vectors, and amplitudes equal up to
    the rounding of the probability sums; the autotuner keeps a valid shape."""
    circuits = c.steane_campaign(64, seed=4) + [c.qft_random_input(8, seed=9)[1]]
    eng = sfm.Campaign(c.STEANE_N, 4096)
    ref = None
    for threads in (32, 64, 128, 256):
        for smem in (True, False):
            try:
                eng.set_shape(threads, smem)
            except sfm.SFError:
                continue
            assert eng.shape()[:2] == (threads, smem)
            res = eng.run(circuits, export=True)
            assert not res["status"].any()
            if ref is None:
                ref = res
                continue
            for key in ("outcomes", "n_meas", "k_final"):
                assert np.array_equal(res[key], ref[key]), (threads, smem, key)
            assert np.max(np.abs(res["norm"] - ref["norm"])) <= 1e-12
            for fa, fb in zip(res["frames"], ref["frames"]):
                assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1]) and fa[2] == fb[2]
                assert np.array_equal(fa[3], fb[3])
                assert np.max(np.abs(fa[4] - fb[4]), initial=0.0) <= 1e-12
    ops, off, nc = eng.upload(circuits)
    ms = eng.autotune(ops, off, nc, reps=1)
    assert ms > 0
    res = eng.run(circuits)
    assert np.array_equal(res["outcomes"], ref["outcomes"])
    eng.close()


@pytest.mark.parametrize("threads", [32, 64, 256])
def test_stage_circuits_vs_oracle(sfm, threads):
    """Stages that branch along new directions, then controlled phases from
    earlier stages' qubits (merges whose partners already exist, after which
    pairs are scattered through the frame) followed by gates that keep the
    pairs: every in-place run must reach the owners of a 64-element window
    beyond its first 32."""
    n = 12
    circuits = [c.stage_circuit(n, 4400 + s, stages=10, per_stage=24) for s in range(4)]
    eng = sfm.Campaign(n, sfm.CAMPAIGN_MAX_ELEMS)
    eng.set_shape(threads, 0)
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        check_against_oracle(res, i, n, ops)
    eng.close()


@pytest.mark.parametrize("threads", [32, 128, 256])
def test_sorted_coalescing_vs_oracle_and_hash(sfm, threads):
    """The sorted coalescing strategy (positions ordered by phase vector, binary
    searches) against the oracle on Steane variants, random Clifford+T circuits,
    the QFT and the stage circuits (frames up to thousands of elements), and bit
    for bit against the hash strategy in the same shape: both find the same
    partners."""
    n = 12
    circuits = ([c.stage_circuit(n, 5100 + s, stages=9, per_stage=20) for s in range(3)] +
                [c.qft_random_input(n, seed=3)[1]] + [c.random_clifford_t(n, 400, 8, seed=21 + i) for i in range(6)])
    eng = sfm.Campaign(n, sfm.CAMPAIGN_MAX_ELEMS)
    eng.set_shape(threads, 0)
    eng.set_coalesce(False)
    ref = eng.run(circuits, export=True)
    eng.set_coalesce(True)
    assert eng.coalesce_sorted()
    res = eng.run(circuits, export=True)
    for i, ops in enumerate(circuits):
        check_against_oracle(res, i, n, ops)
    for key in ("outcomes", "n_meas", "k_final", "status"):
        assert np.array_equal(res[key], ref[key]), key
    assert np.array_equal(res["norm"], ref["norm"])
    for fa, fb in zip(res["frames"], ref["frames"]):
        for a, b in zip(fa, fb):
            assert np.array_equal(np.asarray(a), np.asarray(b))
    eng.close()
    steane = c.steane_campaign(48, seed=6)
    eng = sfm.Campaign(c.STEANE_N, 4096)
    eng.set_coalesce(True)
    res = eng.run(steane, export=True)
    for i, ops in enumerate(steane):
        check_against_oracle(res, i, c.STEANE_N, ops)
    eng.close()


def test_autotuner_searches_both_strategies(sfm):
    """The autotuner times every shape with each strategy and keeps one; the
    kept configuration reproduces the results."""
    circuits = c.steane_campaign(96, seed=8)
    eng = sfm.Campaign(c.STEANE_N, 4096)
    ref = eng.run(circuits)
    ops, off, nc = eng.upload(circuits)
    ms = eng.autotune(ops, off, nc, reps=1)
    assert ms > 0
    assert eng.coalesce_sorted() in (False, True)
    res = eng.run(circuits)
    assert np.array_equal(res["outcomes"], ref["outcomes"])
    assert np.array_equal(res["k_final"], ref["k_final"])
    eng.close()
