"""Host-side checks of the batched-campaign workload (no GPU): the Steane
[[7,1,3]] fault-injection generator is pinned through the oracle against
coding-theory facts, and the program encoding of the campaign ABI is checked
field by field."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_03554_gb300 import circuits as c


def _draws(ops, u=0.5):
    return [("M", op[1], u) if op[0] == "M" else op for op in ops]


def _measure_qubits(ops):
    return [op[1] for op in ops if op[0] == "M"]


def test_steane_layout_uses_49_distinct_qubits():
    L = c.steane_layout()
    qs = list(L["data"]) + [L["magic"], L["read_x"], L["read_z"]] + list(L["checks"])
    for a, f in L["synd"].values():
        qs += [a, f]
    assert sorted(qs) == list(range(c.STEANE_N))


def test_steane_checks_form_the_hamming_code():
    """Each qubit j has the syndrome column j + 1 (binary), the three checks
    pairwise overlap in two qubits (the X and Z stabilizers commute), and the
    logical support {0, 1, 2} has even overlap with every check."""
    for j in range(7):
        col = sum(((j in sup) << (2 - s)) for s, sup in enumerate(c.STEANE_CHECKS))
        assert col == j + 1
    for a in c.STEANE_CHECKS:
        for b in c.STEANE_CHECKS:
            assert len(set(a) & set(b)) % 2 == 0
        assert len(set(a) & set(c.STEANE_LOGICAL)) % 2 == 0


def test_steane_base_without_faults():
    """No error: every syndrome and flag outcome is 0 with certainty; the magic
    measurement is 50/50; after T_L on |+>_L the logical-X readout gives -1 with
    probability (1 - cos(pi/4)) / 2 in either branch of the magic outcome (the
    S_L correction fixes T-dagger to T); the logical-Z readout is 50/50."""
    base = c.steane_base()
    qs = _measure_qubits(base)
    L = c.steane_layout()
    for u in (0.25, 0.75):  # both outcomes of the magic measurement
        o = oracle.FrameOracle(c.STEANE_N)
        res = c.run(o, _draws(base, u))
        assert len(res) == len(qs) == 42
        for (q, p0, p1, x) in res:
            if q == L["magic"]:
                assert abs(p1 - 0.5) < 1e-12
            elif q == L["read_x"]:
                assert abs(p1 - (1 - math.cos(math.pi / 4)) / 2) < 1e-12
            elif q == L["read_z"]:
                assert abs(p1 - 0.5) < 1e-12
            else:
                assert p1 < 1e-12 and x == 0, q
        x_magic = [r[3] for r in res if r[0] == L["magic"]][0]
        assert x_magic == (1 if u < 0.5 else 0)


@pytest.mark.parametrize("j", range(7))
@pytest.mark.parametrize("pauli", [c.X, c.Z, c.Y])
def test_steane_single_error_syndrome(j, pauli):
    """A Pauli error on data qubit j before round 0: X (or Y) flips the Z-type
    checks containing j, Z (or Y) flips the X-type checks containing j -- the
    Hamming syndrome j + 1 -- and the flags stay 0.  Later rounds repeat the
    syndrome (the error is not corrected)."""
    base = c.steane_base()
    L = c.steane_layout()
    a0, f0 = L["synd"][(0, 0)]
    first_round = next(i for i, op in enumerate(base) if op[0] == "C" and f0 in op[2:4])  # flag of round 0 set up
    ops = base[:first_round] + [("C", pauli, j, 0)] + base[first_round:]
    res = c.run(oracle.FrameOracle(c.STEANE_N), _draws(ops, 0.9))
    out = {r[0]: r for r in res}
    for s in range(6):
        a, f = L["synd"][(0, s)]
        detects = (pauli in (c.X, c.Y)) if s < 3 else (pauli in (c.Z, c.Y))
        expect = int(detects and j in c.STEANE_CHECKS[s % 3])
        assert out[a][3] == expect and (out[a][2] > 0.5) == bool(expect), (s, out[a])
        assert out[f][3] == 0 and out[f][2] < 1e-12


def test_conditional_op_follows_parity():
    """("Q", kind, q0, q1, mask) applies iff parity(outcomes & mask) = 1."""
    ops = [("C", c.X, 0, 0), ("M", 0, 0.5), ("C", c.H, 3, 0), ("M", 3, 0.9),
           ("Q", c.X, 1, 0, 0b01), ("Q", c.X, 2, 0, 0b11), ("M", 1, 0.5), ("M", 2, 0.5)]
    o = oracle.FrameOracle(4)
    res = c.run(o, ops)
    assert [r[3] for r in res] == [1, 0, 1, 1]
    ops[3] = ("M", 3, 0.1)  # outcome 1 on qubit 3: parity of 0b11 is now 0
    res = c.run(oracle.FrameOracle(4), ops)
    assert [r[3] for r in res] == [1, 1, 1, 0]


def test_variant_recipe():
    for v in range(20):
        ops = c.steane_variant(v)
        n = c.count_ops(ops)
        assert 200 <= c._gate_count(ops) <= 2001
        assert n["M"] == 42 and n["Q"] == 7
        assert 1 <= n["N"] <= 13
        for i, op in enumerate(ops):
            if op[0] == "N":
                assert ops[i + 1] == ("K",)
            if op[0] == "M":
                assert 0.0 <= op[2] < 1.0
            for q in op[1:4] if op[0] in ("C", "Q") else ():
                assert 0 <= q < c.STEANE_N
    assert c.steane_variant(5) == c.steane_variant(5)
    assert c.steane_variant(5) != c.steane_variant(6)


def test_encode_program_fields():
    from paper_1712_03554_gb300 import sf
    circuits = [[("C", c.CNOT, 3, 4), ("N", c.CPHASE, 1, 2, 0.25), ("K",), ("M", 5, 0.125),
                 ("Q", c.SDG, 6, 0, (1 << 63) | 5)], [], [("N", c.T, 0, 0, 0.0)]]
    rec, off = sf.encode_program(circuits)
    assert rec.dtype.itemsize == 24 and list(off) == [0, 4, 4, 5]
    assert tuple(rec[0])[:4] == (c.CNOT, 3, 4, 0)
    assert tuple(rec[1])[:4] == (sf.OP_DIAG + c.CPHASE, 1, 2, 0) and rec[1]["param"] == 0.25
    assert tuple(rec[2])[:2] == (sf.OP_MEASURE, 5) and rec[2]["param"] == 0.125
    assert tuple(rec[3])[:4] == (sf.OP_COND, 6, 0, c.SDG)
    assert np.array([rec[3]["param"]]).view(np.uint64)[0] == (1 << 63) | 5
    assert tuple(rec[4])[:2] == (sf.OP_DIAG + c.T, 0)
    with pytest.raises(ValueError):
        sf.encode_program([[("M", 0, None)]])


def test_serving_stream_recipe():
    st = c.serving_stream(40, 10.0, seed=3)
    arr = [r["arrival"] for r in st]
    assert all(b > a for a, b in zip(arr, arr[1:]))
    assert {r["n"] for r in st} <= set(c.SERVING_QUBITS)
    for r in st:
        n_c = sum(1 for op in r["ops"] if op[0] == "C")
        n_t = sum(1 for op in r["ops"] if op[0] == "N")
        assert 1000 <= n_c <= 100000 and 0 <= n_t <= 20
        assert r["max_elems"] == 1 << min(n_t + 1, r["n"] + 1, 21)
        assert [op[0] for op in r["ops"][-8:]] == ["M"] * 8 and len({op[1] for op in r["ops"][-8:]}) == 8
        assert r["probes"][0] == 0 and all(0 <= p < (1 << r["n"]) for p in r["probes"])
    assert c.serving_stream(5, 1.0, seed=1)[3]["ops"] == c.serving_stream(5, 1.0, seed=1)[3]["ops"]


def test_server_abi_struct_layouts():
    import ctypes
    from paper_1712_03554_gb300 import sf
    assert ctypes.sizeof(sf.sf_request) == 48
    assert ctypes.sizeof(sf.sf_result) == 128
    assert ctypes.sizeof(sf.sf_server_stats) == 32
    assert sf.SF_OP_DTYPE.itemsize == 24
