"""Seeded synthetic circuit generators and a simulator-agnostic driver.

This module holds no simulation arithmetic: it only builds gate lists (plain
Python tuples) from a seed and walks them against any object exposing the
stabilizer-frame calls (``apply_clifford``, ``apply_nonclifford``,
``coalesce``, ``measure``).  Both the CUDA path and the CPU oracle are driven
through it, so the two always see the same inputs.

Op encoding (one tuple per op):
  ("C", kind, q0, q1)              Clifford gate, kind in CLIFFORD_KINDS
  ("N", kind, q0, q1, theta)       diagonal non-Clifford gate, kind in NONCLIFFORD_KINDS
  ("K",)                           coalesce the frame
  ("M", q, u)                      measure qubit q; outcome = 1 if u < p(1) else 0
                                   (u is a seeded uniform draw, or None for
                                   "probabilities only")
  ("T3", c1, c2, t)                Toffoli by cofactors (Eq. 2): COFACTOR on c1, c2,
                                   X_t on the 11 cofactor
  ("CR", c, t, alpha)              controlled-R(alpha) by cofactors (Eq. 3)
  ("Q", kind, q0, q1, mask)        classically controlled Clifford gate: applied
                                   iff the parity of (outcome bits & mask) is 1,
                                   bit m = outcome of the m-th drawn measurement

Gate semantics follow the paper: H, P (= S) and CNOT are the Clifford gates of
Table 2 (Sec. II-B); T/T-dagger are the technology-dependent non-Clifford gates
of Sec. IV; controlled-R(alpha) is Eq. 3.  The Toffoli is expanded into
Clifford+T as the paper does for its "Clifford+T" rows (Sec. VI, Toffoli
decomposition), using the textbook 7-T network.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

# ---- gate kind codes (must match include/sf.h) --------------------------------
H, S, SDG, X, Y, Z, CNOT, CZ, SWAP = range(9)
CLIFFORD_KINDS = {"H": H, "S": S, "SDG": SDG, "X": X, "Y": Y, "Z": Z,
                  "CNOT": CNOT, "CZ": CZ, "SWAP": SWAP}
TWO_QUBIT_CLIFFORD = {CNOT, CZ, SWAP}
T, TDG, PHASE, CPHASE = range(4)
NONCLIFFORD_KINDS = {"T": T, "TDG": TDG, "PHASE": PHASE, "CPHASE": CPHASE}

Op = Tuple


def rng_for(seed: int) -> np.random.Generator:
    """Every workload draws from numpy's PCG64 seeded with an integer."""
    return np.random.Generator(np.random.PCG64(seed))


# ---- building blocks ------------------------------------------------------------
def toffoli_clifford_t(a: int, b: int, c: int) -> List[Op]:
    """Toffoli(controls a, b; target c) as 2 H + 6 CNOT + 7 T/T-dagger.

    The textbook network (the decomposition the paper's "Clifford+T" table rows
    use, Sec. VI).  Its 8x8 unitary is checked against the Toffoli in the dense
    oracle tests.
    """
    return [
        ("C", H, c, 0),
        ("C", CNOT, b, c), ("N", TDG, c, 0, 0.0),
        ("C", CNOT, a, c), ("N", T, c, 0, 0.0),
        ("C", CNOT, b, c), ("N", TDG, c, 0, 0.0),
        ("C", CNOT, a, c), ("N", T, b, 0, 0.0), ("N", T, c, 0, 0.0),
        ("C", H, c, 0),
        ("C", CNOT, a, b), ("N", T, a, 0, 0.0), ("N", TDG, b, 0, 0.0),
        ("C", CNOT, a, b),
    ]


def with_coalesce_after_nonclifford(ops: Sequence[Op]) -> List[Op]:
    out: List[Op] = []
    for op in ops:
        out.append(op)
        if op[0] == "N":
            out.append(("K",))
    return out


# ---- workload 1: random Clifford+T on 8 qubits ------------------------------------
def random_clifford_t(n: int = 8, n_gates: int = 200, n_t: int = 4, seed: int = 0,
                      t_kinds: Sequence[int] = (T,)) -> List[Op]:
    """n qubits from |0..0>, n_gates gates of which exactly n_t are T at distinct
    uniform positions; the rest uniform over {H, S, CNOT}, one-qubit targets
    uniform over the qubits, CNOT ordered pairs uniform over the n(n-1) pairs.
    A coalesce follows every T."""
    g = rng_for(seed)
    t_pos = set(int(p) for p in g.choice(n_gates, size=n_t, replace=False))
    ops: List[Op] = []
    for i in range(n_gates):
        if i in t_pos:
            kind = t_kinds[int(g.integers(len(t_kinds)))]
            ops.append(("N", kind, int(g.integers(n)), 0, 0.0))
            ops.append(("K",))
            continue
        kind = (H, S, CNOT)[int(g.integers(3))]
        if kind == CNOT and n >= 2:
            c = int(g.integers(n))
            t = int(g.integers(n - 1))
            t = t + 1 if t >= c else t
            ops.append(("C", CNOT, c, t))
        else:
            ops.append(("C", kind if kind != CNOT else H, int(g.integers(n)), 0))
    return ops


def random_clifford(n: int, n_gates: int, seed: int,
                    kinds: Sequence[int] = (H, S, CNOT)) -> List[Op]:
    """Random stabilizer circuit over the given Clifford kinds (no non-Clifford)."""
    g = rng_for(seed)
    ops: List[Op] = []
    for _ in range(n_gates):
        kind = kinds[int(g.integers(len(kinds)))]
        if kind in TWO_QUBIT_CLIFFORD:
            if n < 2:
                continue
            c = int(g.integers(n))
            t = int(g.integers(n - 1))
            t = t + 1 if t >= c else t
            ops.append(("C", kind, c, t))
        else:
            ops.append(("C", kind, int(g.integers(n)), 0))
    return ops


# ---- workload 2: QFT on a basis state ------------------------------------------------
def qft_phase(k: int) -> float:
    """R_k = diag(1, exp(2 pi i / 2^k)); k = distance + 1 (paper Sec. VI, QFT)."""
    return 2.0 * math.pi / float(1 << k) if k < 1024 else 0.0


def qft(n: int, x: int, coalesce: bool = True) -> List[Op]:
    """X gates prepare |x> (bit q of x is qubit q), then the swap-free QFT:
    for j = 0..n-1: H on j, then controlled-R_k (k = 2..n-j) with control
    j+k-1 and target j.  n(n+1)/2 gates after the preparation."""
    ops: List[Op] = [("C", X, q, 0) for q in range(n) if (x >> q) & 1]
    for j in range(n):
        ops.append(("C", H, j, 0))
        for k in range(2, n - j + 1):
            ops.append(("N", CPHASE, j + k - 1, j, qft_phase(k)))
            if coalesce:
                ops.append(("K",))
    return ops


def qft_random_input(n: int = 20, seed: int = 0) -> Tuple[int, List[Op]]:
    g = rng_for(seed)
    x = int(g.integers(0, 1 << n)) if n < 63 else int(g.integers(0, 1 << 62))
    return x, qft(n, x)


def qft_expected_amplitude(n: int, x: int, y: int) -> complex:
    """Closed form of the swap-free QFT output (Sec. VI, QFT equation), read
    with qubit j (0-based, the j-th to get its H) ending in
    (|0> + exp(2 pi i 0.x_j x_{j+1} ... x_{n-1}) |1>)/sqrt(2), where x_j is bit j of x."""
    amp = 1.0 + 0.0j
    for j in range(n):
        frac = 0.0
        for m, q in enumerate(range(j, n)):
            if (x >> q) & 1:
                frac += 2.0 ** (-(m + 1))
        if (y >> j) & 1:
            amp *= complex(math.cos(2 * math.pi * frac), math.sin(2 * math.pi * frac))
    return amp / math.sqrt(2.0 ** n)


# ---- workload 3: Cuccaro ripple-carry adder -------------------------------------------
def stage_circuit(n: int, seed: int, stages: int, per_stage: int) -> List[Op]:
    """Stages shaped like the QFT's: X on random qubits, then per stage H on a
    fresh target t and a run of controlled phases onto t from random other
    qubits (angles pi/2, pi, pi/4, -pi/2, 2 pi/3: exact zeros when a control
    is |0>, cancellations when angles add up to multiples of 2 pi), T and
    T-dagger on t, and one-qubit phases on random qubits.  Each stage branches
    along a new direction; controls from earlier stages make merges whose
    partners already exist."""
    g = rng_for(seed)
    ops: List[Op] = [("C", X, q, 0) for q in range(n) if g.random() < 0.5]
    for s in range(stages):
        t = s % n
        ops.append(("C", H, t, 0))
        for _ in range(per_stage):
            r = g.random()
            if r < 0.6:
                ctl = int(g.integers(n - 1))
                ctl += ctl >= t
                th = float(g.choice([np.pi / 2, np.pi, np.pi / 4, -np.pi / 2, 2 * np.pi / 3]))
                ops += [("N", CPHASE, ctl, t, th), ("K",)]
            elif r < 0.8:
                ops += [("N", T if g.random() < 0.5 else TDG, t, 0, 0.0), ("K",)]
            else:
                q = int(g.integers(n))
                ops += [("N", PHASE, q, 0, float(g.uniform(-3, 3))), ("K",)]
    return ops


def cuccaro_layout(nbits: int):
    """Qubit 0 = ancilla (carry-in), then interleaved b_i, a_i for i = 0..nbits-1,
    then the carry-out z.  Returns (anc, a[], b[], z)."""
    anc = 0
    b = [1 + 2 * i for i in range(nbits)]
    a = [2 + 2 * i for i in range(nbits)]
    z = 2 * nbits + 1
    return anc, a, b, z


def cuccaro_classical_ops(nbits: int):
    """The reversible network as ('cnot', c, t) / ('tof', c1, c2, t) records:
    MAJ blocks up the chain, a CNOT into the carry, UMA blocks down."""
    anc, a, b, z = cuccaro_layout(nbits)
    net = []

    def maj(c, bb, aa):
        net.extend([("cnot", aa, bb), ("cnot", aa, c), ("tof", c, bb, aa)])

    def uma(c, bb, aa):
        net.extend([("tof", c, bb, aa), ("cnot", aa, c), ("cnot", c, bb)])

    maj(anc, b[0], a[0])
    for i in range(1, nbits):
        maj(a[i - 1], b[i], a[i])
    net.append(("cnot", a[nbits - 1], z))
    for i in range(nbits - 1, 0, -1):
        uma(a[i - 1], b[i], a[i])
    uma(anc, b[0], a[0])
    return net


def cuccaro(nbits: int, superpose: bool = True, a_val: int = 0, b_val: int = 0,
            coalesce: bool = True, toffoli: str = "clifford_t") -> List[Op]:
    """Cuccaro adder with every Toffoli as Clifford+7T (toffoli="clifford_t") or
    applied directly by cofactors, Eq. 2 (toffoli="cofactor").  With
    superpose=True the inputs are H on every a and b qubit (the paper's
    benchmark, Sec. VI); otherwise X gates load the basis inputs a_val, b_val."""
    anc, a, b, z = cuccaro_layout(nbits)
    ops: List[Op] = []
    if superpose:
        ops += [("C", H, q, 0) for q in a + b]
    else:
        ops += [("C", X, a[i], 0) for i in range(nbits) if (a_val >> i) & 1]
        ops += [("C", X, b[i], 0) for i in range(nbits) if (b_val >> i) & 1]
    for rec in cuccaro_classical_ops(nbits):
        if rec[0] == "cnot":
            ops.append(("C", CNOT, rec[1], rec[2]))
        elif toffoli == "cofactor":
            ops.append(("T3", rec[1], rec[2], rec[3]))
        else:
            ops += toffoli_clifford_t(rec[1], rec[2], rec[3])
    return with_coalesce_after_nonclifford(ops) if coalesce else ops


def cuccaro_reference(nbits: int, a_val: int, b_val: int) -> int:
    """Run the reversible network on classical bits; return the output basis index."""
    anc, a, b, z = cuccaro_layout(nbits)
    nq = 2 * nbits + 2
    bits = [0] * nq
    for i in range(nbits):
        bits[a[i]] = (a_val >> i) & 1
        bits[b[i]] = (b_val >> i) & 1
    for rec in cuccaro_classical_ops(nbits):
        if rec[0] == "cnot":
            bits[rec[2]] ^= bits[rec[1]]
        else:
            bits[rec[3]] ^= bits[rec[1]] & bits[rec[2]]
    return sum(bit << q for q, bit in enumerate(bits))


def cuccaro_sample_ops(nbits: int, seed: int) -> List[Op]:
    """Measure every qubit in order with seeded uniform draws (sampling)."""
    g = rng_for(seed)
    return [("M", q, float(g.random())) for q in range(2 * nbits + 2)]


# ---- driver ------------------------------------------------------------------------
def run(sim, ops: Sequence[Op], drop_eps: float = 1e-12, batch_cliffords: bool = True,
        outcome_bits: int = 0, n_drawn: int = 0):
    """Walk ops against sim.  Consecutive Clifford gates are passed as one batch;
    a non-Clifford gate directly followed by a coalesce goes to
    sim.apply_nonclifford_coalesce when sim has it.  Returns the list of
    (q, p0, p1, outcome) for every measurement.  outcome_bits / n_drawn carry
    the outcomes of measurements already made on sim (for conditional gates)
    when a circuit is continued from the middle."""
    pending: List[Tuple[int, int, int]] = []
    results = []

    def flush():
        if pending:
            sim.apply_clifford(list(pending))
            pending.clear()

    fused = getattr(sim, "apply_nonclifford_coalesce", None)
    skip_next = False
    for i, op in enumerate(ops):
        if skip_next:
            skip_next = False
            continue
        tag = op[0]
        if tag == "C":
            pending.append((op[1], op[2], op[3]))
            if not batch_cliffords:
                flush()
        elif tag == "N":
            flush()
            if fused is not None and i + 1 < len(ops) and ops[i + 1][0] == "K":
                fused(op[1], op[2], op[3], op[4], drop_eps)  # branch and merge in one call
                skip_next = True
            else:
                sim.apply_nonclifford(op[1], op[2], op[3], op[4])
        elif tag == "K":
            flush()
            sim.coalesce(drop_eps)
        elif tag == "M":
            flush()
            q, u = op[1], op[2]
            p0, p1 = sim.measure(q, -1)
            if u is None:
                results.append((q, p0, p1, None))
            else:
                x = 1 if u < p1 else 0
                sim.measure(q, x)
                results.append((q, p0, p1, x))
                outcome_bits |= x << n_drawn
                n_drawn += 1
        elif tag == "T3":
            flush()
            sim.apply_toffoli_cofactor(op[1], op[2], op[3])
        elif tag == "CR":
            flush()
            sim.apply_cr_cofactor(op[1], op[2], op[3])
        elif tag == "Q":
            if bin(outcome_bits & op[4]).count("1") & 1:
                pending.append((op[1], op[2], op[3]))
                if not batch_cliffords:
                    flush()
        else:
            raise ValueError(f"unknown op {op!r}")
    flush()
    return results


# ---- workload 4: Steane [[7,1,3]] fault-injection campaign ---------------------------
# Hamming [7,4] parity checks; each support carries one X-type and one Z-type
# stabilizer of the Steane code.  {0, 1, 2} is a weight-3 Hamming codeword, so
# X and Z on qubits 0, 1, 2 are logical X and Z representatives.
STEANE_CHECKS = ((3, 4, 5, 6), (1, 2, 5, 6), (0, 2, 4, 6))
STEANE_LOGICAL = (0, 1, 2)
STEANE_N = 49
STEANE_ROUNDS = 3
INVERSE_CLIFFORD = {H: H, S: SDG, SDG: S, X: X, Y: Y, Z: Z, CNOT: CNOT, CZ: CZ, SWAP: SWAP}


def steane_layout():
    """Qubit roles of the 49-qubit campaign circuit: data 0..6, magic-state
    ancilla 7; for round r and stabilizer s (0..2 Z-type, 3..5 X-type) a
    syndrome ancilla 8 + 12 r + 2 s and its flag 9 + 12 r + 2 s; readout
    ancillas 44 (logical X), 45 (logical Z), 46..48 (final Z checks)."""
    synd = {(r, s): (8 + 12 * r + 2 * s, 9 + 12 * r + 2 * s) for r in range(STEANE_ROUNDS) for s in range(6)}
    return {"data": list(range(7)), "magic": 7, "synd": synd, "read_x": 44, "read_z": 45,
            "checks": [46, 47, 48]}


def _stabilizer_round(r: int, L) -> List[Op]:
    """One flagged syndrome-extraction round: each weight-4 stabilizer is read
    through one ancilla, with a flag qubit coupled between the first and the
    last data CNOT."""
    ops: List[Op] = []
    for s in range(6):
        a, f = L["synd"][(r, s)]
        sup = STEANE_CHECKS[s % 3]
        if s < 3:  # Z-type: data -> ancilla parity; flag in |+>, X-basis readout
            ops += [("C", H, f, 0), ("C", CNOT, sup[0], a), ("C", CNOT, f, a), ("C", CNOT, sup[1], a),
                    ("C", CNOT, sup[2], a), ("C", CNOT, f, a), ("C", CNOT, sup[3], a), ("C", H, f, 0),
                    ("M", f, None), ("M", a, None)]
        else:      # X-type: ancilla in |+> drives the data; flag in |0>
            ops += [("C", H, a, 0), ("C", CNOT, a, sup[0]), ("C", CNOT, a, f), ("C", CNOT, a, sup[1]),
                    ("C", CNOT, a, sup[2]), ("C", CNOT, a, f), ("C", CNOT, a, sup[3]), ("C", H, a, 0),
                    ("M", a, None), ("M", f, None)]
    return ops


def steane_base() -> List[Op]:
    """Encode |0>_L, transversal H (|+>_L), syndrome round 0, logical T by an
    injected magic state (ancilla 7 in T|+>, CNOTs from the logical-Z support,
    measure; outcome 1 -> S_L, which for the Steane code is S-dagger on every
    data qubit), rounds 1..2, then logical X and Z readouts and three final
    Z checks.  Measurement draws are left as None."""
    L = steane_layout()
    ops: List[Op] = [("C", H, 0, 0), ("C", H, 1, 0), ("C", H, 3, 0)]
    for src, tgts in ((0, (2, 4, 6)), (1, (2, 5, 6)), (3, (4, 5, 6))):
        ops += [("C", CNOT, src, t) for t in tgts]
    ops += [("C", H, q, 0) for q in L["data"]]
    ops += _stabilizer_round(0, L)
    m = L["magic"]
    ops += [("C", H, m, 0), ("N", T, m, 0, 0.0), ("K",)]
    ops += [("C", CNOT, q, m) for q in STEANE_LOGICAL]
    ops += [("M", m, None), ("QT",)]  # ("QT",): conditional S_L on the magic outcome, resolved below
    for r in range(1, STEANE_ROUNDS):
        ops += _stabilizer_round(r, L)
    rx, rz = L["read_x"], L["read_z"]
    ops += [("C", H, rx, 0)] + [("C", CNOT, rx, q) for q in STEANE_LOGICAL] + [("C", H, rx, 0), ("M", rx, None)]
    ops += [("C", CNOT, q, rz) for q in STEANE_LOGICAL] + [("M", rz, None)]
    for c, sup in zip(L["checks"], STEANE_CHECKS):
        ops += [("C", CNOT, q, c) for q in sup] + [("M", c, None)]
    # resolve the conditional correction: mask = bit of the magic measurement
    out: List[Op] = []
    n_meas = 0
    for op in ops:
        if op[0] == "M":
            n_meas += 1
        if op[0] == "QT":
            out += [("Q", SDG, q, 0, 1 << (n_meas - 1)) for q in L["data"]]
        else:
            out.append(op)
    return out


def _gate_count(ops: Sequence[Op]) -> int:
    return sum(1 for op in ops if op[0] != "K")


def steane_variant(seed: int, min_len: int = 200, max_len: int = 2000, max_coherent: int = 12) -> List[Op]:
    """One fault-injection variant of steane_base(): 1-3 single-qubit Pauli
    errors (X, Y or Z) on uniform qubits at uniform positions, t_v uniform in
    0..max_coherent coherent T or T-dagger faults on uniform data qubits at
    uniform positions, padding with adjacent (g, g^-1) Clifford pairs on
    uniform qubits to a length drawn uniform in [min_len, max_len] (ops other
    than coalesces), and a uniform draw for every measurement."""
    g = rng_for(seed)
    base = steane_base()
    n = STEANE_N
    # insertion points: before base op i (i = len(base): at the end), never
    # between an ("N", ...) and its ("K",)
    pts = [i for i in range(len(base) + 1) if not (i < len(base) and base[i][0] == "K")]
    buckets: List[List[Op]] = [[] for _ in range(len(base) + 1)]
    count = _gate_count(base)

    def insert(seq):
        nonlocal count
        buckets[pts[int(g.integers(len(pts)))]].extend(seq)
        count += _gate_count(seq)

    for _ in range(int(g.integers(1, 4))):
        insert([("C", (X, Y, Z)[int(g.integers(3))], int(g.integers(n)), 0)])
    for _ in range(int(g.integers(0, max_coherent + 1))):
        insert([("N", (T, TDG)[int(g.integers(2))], int(g.integers(7)), 0, 0.0), ("K",)])
    target = int(g.integers(min_len, max_len + 1))
    n_pairs = max(0, (target - count + 1) // 2)
    kinds = (H, S, SDG, X, Y, Z, CNOT, CZ, SWAP)
    ks = g.integers(len(kinds), size=n_pairs)
    qa = g.integers(n, size=n_pairs)
    qb = g.integers(n - 1, size=n_pairs)
    at = g.integers(len(pts), size=n_pairs)
    for k_i, a, b, p in zip(ks.tolist(), qa.tolist(), qb.tolist(), at.tolist()):
        k = kinds[k_i]
        if k in TWO_QUBIT_CLIFFORD:
            b = b + 1 if b >= a else b
            buckets[pts[p]] += [("C", k, a, b), ("C", INVERSE_CLIFFORD[k], a, b)]
        else:
            buckets[pts[p]] += [("C", k, a, 0), ("C", INVERSE_CLIFFORD[k], a, 0)]
    ops: List[Op] = []
    for i in range(len(base) + 1):
        ops.extend(buckets[i])
        if i < len(base):
            ops.append(base[i])
    return [("M", op[1], float(g.random())) if op[0] == "M" else op for op in ops]


def steane_campaign(n_variants: int = 4096, seed: int = 0, **kw) -> List[List[Op]]:
    """n_variants seeded variants (variant v uses seed * 1_000_003 + v)."""
    return [steane_variant(seed * 1_000_003 + v, **kw) for v in range(n_variants)]


# ---- workload 5: a Poisson stream of served circuits ---------------------------------
SERVING_QUBITS = (16, 64, 256, 1024)


def serving_circuit(seed: int, n: int, n_cliff: int, n_t: int) -> List[Op]:
    """Random Clifford+T circuit: n_cliff gates uniform over {H, S, CNOT} (one-
    qubit targets and ordered CNOT pairs uniform), n_t T gates at uniform
    positions on uniform qubits, each followed by a coalesce."""
    g = rng_for(seed)
    kinds = g.integers(3, size=n_cliff)
    qa = g.integers(n, size=n_cliff)
    qb = g.integers(max(n - 1, 1), size=n_cliff)
    ops: List[Op] = []
    for k, a, b in zip(kinds.tolist(), qa.tolist(), qb.tolist()):
        if k == 2 and n > 1:
            ops.append(("C", CNOT, a, b + 1 if b >= a else b))
        else:
            ops.append(("C", (H, S, H)[k], a, 0))
    t_pos = sorted(g.choice(n_cliff + 1, size=n_t, replace=True).tolist(), reverse=True)
    t_q = g.integers(n, size=n_t).tolist()
    for p, q in zip(t_pos, t_q):
        ops[p:p] = [("N", T, q, 0, 0.0), ("K",)]
    return ops


def serving_stream(n_requests: int, rate_hz: float, seed: int = 0, qubits: Sequence[int] = SERVING_QUBITS,
                   cliff_range=(1000, 100000), max_t: int = 20, n_probes: int = 4, n_measure: int = 8):
    """A seeded Poisson stream of requests: exponential inter-arrival times of
    mean 1/rate_hz; n uniform over `qubits`; the Clifford count log-uniform in
    cliff_range; the T count uniform in 0..max_t; frame capacity
    2^min(T, n + 1, 20) (each T at most doubles the frame, and a frame on n
    qubits holds at most 2^n elements before a branch doubles it); probes:
    |0...0> and uniform basis states.  Returns dicts with arrival (s), n, ops,
    max_elems, probes."""
    g = rng_for(seed)
    t = 0.0
    out = []
    lo, hi = math.log(cliff_range[0]), math.log(cliff_range[1])
    for i in range(n_requests):
        t += float(g.exponential(1.0 / rate_hz))
        n = int(qubits[int(g.integers(len(qubits)))])
        n_cliff = int(round(math.exp(g.uniform(lo, hi))))
        n_t = int(g.integers(0, max_t + 1))
        probes = [0] + [int(x) for x in (int(g.integers(1 << 62)) for _ in range(n_probes - 1))]
        probes = [p & ((1 << n) - 1) for p in probes]
        ops = serving_circuit(seed * 7919 + i, n, n_cliff, n_t)
        mq = g.choice(n, size=min(n_measure, n), replace=False).tolist()
        ops += [("M", int(q), float(g.random())) for q in mq]
        out.append({"arrival": t, "n": n, "ops": ops,
                    "max_elems": 1 << min(n_t + 1, n + 1, 21), "probes": probes})
    return out


def count_ops(ops: Sequence[Op]):
    c = {"C": 0, "N": 0, "K": 0, "M": 0, "Q": 0, "T3": 0, "CR": 0}
    for op in ops:
        c[op[0]] += 1
    return c
