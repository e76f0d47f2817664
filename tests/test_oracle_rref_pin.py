"""Pin of the oracle's Gauss-Jordan elimination (Invariant 1, Sec. III) at
word boundaries, by a second elimination written here from the definitions.

The stabilizer group after a Clifford circuit is found without the oracle's
tables: each unsigned row (x | z) is conjugated by the binary symplectic rules
of the gates (H swaps x_q and z_q; S and S-dagger add x_q to z_q; CNOT c->t
adds x_c to x_t and z_t to z_c; CZ adds x_b to z_a and x_a to z_b; SWAP swaps
the two qubits; Pauli gates change signs only), and a random-outcome
measurement of q replaces the group by the rows commuting with Z_q plus Z_q
(Sec. II-B).  The rows are then brought to reduced row-echelon form over the
columns x_0..x_{n-1}, z_0..z_{n-1} (each row a 2n-bit integer with column 0
most significant, reduced with a pivot per leading bit).  The RREF of a row
space is unique, so the oracle's tableau must equal it row for row, together
with the X-block size (rows whose pivot is an x column).
"""
import numpy as np
import pytest

import oracle

H, S, SDG, X, Y, Z, CNOT, CZ, SWAP = range(9)


def _bit(v, q):
    return (v >> q) & 1


def _conj(rows, kind, a, b):
    out = []
    for x, z in rows:
        if kind == H:
            xa, za = _bit(x, a), _bit(z, a)
            x ^= (xa ^ za) << a
            z ^= (xa ^ za) << a
        elif kind in (S, SDG):
            z ^= _bit(x, a) << a
        elif kind == CNOT:
            x ^= _bit(x, a) << b
            z ^= _bit(z, b) << a
        elif kind == CZ:
            z ^= (_bit(x, b) << a) ^ (_bit(x, a) << b)
        elif kind == SWAP:
            for v in ("x", "z"):
                w = x if v == "x" else z
                if _bit(w, a) != _bit(w, b):
                    w ^= (1 << a) | (1 << b)
                if v == "x":
                    x = w
                else:
                    z = w
        out.append((x, z))
    return out


def _measure(rows, n, q):
    """Unsigned stabilizer group after a random-outcome measurement of q."""
    anti = [i for i, (x, z) in enumerate(rows) if _bit(x, q)]
    if not anti:
        return rows
    p = anti[0]
    px, pz = rows[p]
    out = list(rows)
    for i in anti[1:]:
        out[i] = (out[i][0] ^ px, out[i][1] ^ pz)
    out[p] = (0, 1 << q)
    return out


def _pack(n, x, z):
    """Row as a 2n-bit integer, column x_0 most significant, z_{n-1} least."""
    v = 0
    for c in range(n):
        v = (v << 1) | _bit(x, c)
    for c in range(n):
        v = (v << 1) | _bit(z, c)
    return v


def _unpack(n, v):
    x = z = 0
    for c in range(n):
        z |= ((v >> (n - 1 - c)) & 1) << c
        x |= ((v >> (2 * n - 1 - c)) & 1) << c
    return x, z


def _rref(n, rows):
    basis = {}
    for x, z in rows:
        v = _pack(n, x, z)
        while v:
            lead = v.bit_length() - 1
            if lead not in basis:
                basis[lead] = v
                break
            v ^= basis[lead]
    assert len(basis) == n  # n independent generators
    leads = sorted(basis, reverse=True)  # ascending column
    for i, li in enumerate(leads):       # clear each pivot column in every other row
        for lj in leads:
            if lj != li and (basis[lj] >> li) & 1:
                basis[lj] ^= basis[li]
    out = [_unpack(n, basis[l]) for l in leads]
    r = sum(1 for l in leads if l >= n)  # pivot in an x column
    return out, r


def _oracle_rows(o, n):
    ox, oz, r = o.tableau()
    rows = []
    for h in range(n):
        x = z = 0
        for w in range(ox.shape[1]):
            x |= int(ox[h, w]) << (64 * w)
            z |= int(oz[h, w]) << (64 * w)
        rows.append((x, z))
    return rows, r


@pytest.mark.parametrize("n", [1, 2, 5, 63, 64, 65, 127, 128, 129, 130])
def test_oracle_rref_equals_independent_elimination(n):
    rng = np.random.Generator(np.random.PCG64(1000 + n))
    o = oracle.FrameOracle(n)
    rows = [(0, 1 << q) for q in range(n)]
    n_gates = 120 if n >= 100 else 200
    checks = 0
    for g in range(n_gates):
        kind = int(rng.integers(9)) if n > 1 else int(rng.integers(6))
        a = int(rng.integers(n))
        b = int(rng.integers(n - 1)) if n > 1 else 0
        b += b >= a
        o.apply_clifford([(kind, a, b if kind >= CNOT else 0)])
        rows = _conj(rows, kind, a, b)
        if g % 17 == 16:  # a measurement now and then: cofactor, then collapse on a likely outcome
            q = int(rng.integers(n))
            p0, p1 = o.measure(q, -1)
            o.measure(q, 0 if p0 >= p1 else 1)
            rows = _measure(rows, n, q)
        if g % 10 == 9 or g == n_gates - 1:
            want, r_want = _rref(n, rows)
            got, r_got = _oracle_rows(o, n)
            assert r_got == r_want, (n, g)
            assert got == want, (n, g)
            rows = want
            checks += 1
    assert checks >= 12


def test_planted_row_difference_is_caught():
    """A tableau that differs from the elimination in one bit fails the pin."""
    n = 65
    rows = [(0, 1 << q) for q in range(n)]
    rows = _conj(rows, H, 3, 0)
    rows = _conj(rows, CNOT, 3, 64)
    want, r = _rref(n, rows)
    o = oracle.FrameOracle(n)
    o.apply_clifford([(H, 3, 0), (CNOT, 3, 64)])
    got, r_got = _oracle_rows(o, n)
    assert got == want and r_got == r
    bad = list(got)
    bad[0] = (bad[0][0], bad[0][1] ^ (1 << 64))
    assert bad != want
