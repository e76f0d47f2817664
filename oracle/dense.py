"""Dense FP64 state-vector oracle (n <= 22).  TEST INFRASTRUCTURE ONLY.

The "straightforward implementation of the state-vector model using an array
of complex amplitudes" that the paper checks its simulator against (Sec. VI).
Basis index b = sum_q b_q 2^q (qubit 0 is the least significant bit).  Gate
matrices are written out here from their textbook definitions; nothing is
shared with the frame oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

_r = 1.0 / math.sqrt(2.0)
ONE_QUBIT = {
    0: np.array([[_r, _r], [_r, -_r]], dtype=complex),   # H
    1: np.array([[1, 0], [0, 1j]], dtype=complex),       # S = P
    2: np.array([[1, 0], [0, -1j]], dtype=complex),      # S^dagger
    3: np.array([[0, 1], [1, 0]], dtype=complex),        # X
    4: np.array([[0, -1j], [1j, 0]], dtype=complex),     # Y
    5: np.array([[1, 0], [0, -1]], dtype=complex),       # Z
}


def two_qubit_matrix(kind: int) -> np.ndarray:
    """4x4 matrix on local index l = bit(q0) + 2 bit(q1), U[out, in]."""
    U = np.zeros((4, 4), dtype=complex)
    for lin in range(4):
        b0, b1 = lin & 1, lin >> 1
        if kind == 6:      # CNOT, control q0, target q1
            U[b0 | ((b1 ^ b0) << 1), lin] = 1
        elif kind == 7:    # CZ
            U[lin, lin] = -1 if (b0 and b1) else 1
        elif kind == 8:    # SWAP
            U[b1 | (b0 << 1), lin] = 1
        else:
            raise ValueError(kind)
    return U


class DenseOracle:
    def __init__(self, n: int):
        if n > 24:
            raise ValueError("dense oracle is limited to small n")
        self.n = n
        self.idx = np.arange(1 << n, dtype=np.int64)
        self.reset()

    def reset(self):
        self.psi = np.zeros(1 << self.n, dtype=complex)
        self.psi[0] = 1.0

    def _apply1(self, U, q):
        n = self.n
        v = self.psi.reshape(1 << (n - q - 1), 2, 1 << q)
        self.psi = np.einsum("ij,ajb->aib", U, v).reshape(-1)

    def _apply2(self, U, q0, q1):
        idx = self.idx
        l = ((idx >> q0) & 1) | (((idx >> q1) & 1) << 1)
        base = idx & ~((1 << q0) | (1 << q1))
        new = np.zeros_like(self.psi)
        for lin in range(4):
            pos = ((lin & 1) << q0) | ((lin >> 1) << q1)
            new += U[l, lin] * self.psi[base | pos]
        self.psi = new

    def apply_clifford(self, gates):
        for g in gates:
            kind, q0, q1 = int(g[0]), int(g[1]), int(g[2])
            if kind in ONE_QUBIT:
                self._apply1(ONE_QUBIT[kind], q0)
            else:
                self._apply2(two_qubit_matrix(kind), q0, q1)

    def apply_nonclifford(self, kind, q0, q1=0, theta=0.0):
        if kind == 0:
            theta, kind = math.pi / 4, 2
        elif kind == 1:
            theta, kind = -math.pi / 4, 2
        ph = complex(math.cos(theta), math.sin(theta))
        if kind == 2:
            mask = ((self.idx >> q0) & 1) == 1
        elif kind == 3:
            mask = (((self.idx >> q0) & 1) == 1) & (((self.idx >> q1) & 1) == 1)
        else:
            raise ValueError(kind)
        self.psi = np.where(mask, self.psi * ph, self.psi)

    def apply_toffoli_cofactor(self, c1, c2, t):
        """The Toffoli gate itself (its definition: flip bit t where bits c1 and
        c2 are 1), the dense counterpart of the cofactor-based frame update."""
        both = (((self.idx >> c1) & 1) & ((self.idx >> c2) & 1)) == 1
        src = np.where(both, self.idx ^ (1 << t), self.idx)
        self.psi = self.psi[src]

    def apply_cr_cofactor(self, c, t, alpha):
        """R(alpha)_{ct} by its definition: e^{i alpha} where bits c and t are 1."""
        self.apply_nonclifford(3, c, t, alpha)

    def coalesce(self, eps=1e-12):
        return None

    def measure(self, q, collapse=-1):
        bit = ((self.idx >> q) & 1) == 1
        pr = np.abs(self.psi) ** 2
        p1 = float(pr[bit].sum())
        p0 = float(pr[~bit].sum())
        if collapse in (0, 1):
            p = p1 if collapse else p0
            keep = bit if collapse else ~bit
            self.psi = np.where(keep, self.psi / math.sqrt(p), 0.0)
        return p0, p1

    def amplitude(self, x: int) -> complex:
        return complex(self.psi[x])

    def state(self) -> np.ndarray:
        return self.psi.copy()


# ---- dense helpers used by the pins ------------------------------------------
PAULI = {0: np.eye(2, dtype=complex),                       # I
         1: np.array([[1, 0], [0, -1]], dtype=complex),     # Z
         2: np.array([[0, 1], [1, 0]], dtype=complex),      # X
         3: np.array([[0, -1j], [1j, 0]], dtype=complex)}   # Y


def pauli_row_matrix(xbits: int, zbits: int, n: int) -> np.ndarray:
    """Dense matrix of the unsigned row (x, z): qubit q carries literal
    (x_q z_q) -> I/Z/X/Y; qubit 0 is the least significant tensor factor."""
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        lit = (((xbits >> q) & 1) << 1) | ((zbits >> q) & 1)
        M = np.kron(M, PAULI[lit])
    return M


def frame_state(n: int, xrows, zrows, sigmas, amps, basis_amp) -> np.ndarray:
    """Expand sum_j a_j psi(M, sigma_j) densely using a per-state amplitude
    function basis_amp(sigma, y)."""
    psi = np.zeros(1 << n, dtype=complex)
    for s, a in zip(sigmas, amps):
        for y in range(1 << n):
            v = basis_amp(s, y)
            if v != 0:
                psi[y] += a * v
    return psi


def stabilizer_state_by_projection(n: int, xrows, zrows, sigma: int) -> np.ndarray:
    """The unit vector stabilized by (-1)^{sigma_h} P(x_h, z_h) for every row,
    built by projecting a basis vector with prod_h (I + (-1)^{s_h} P_h)/2 and
    fixing the phase so that the amplitude at the anchor (the support element
    with zero bits at every X-pivot qubit) is real and positive.  Independent of
    the frame oracle's closed form."""
    dim = 1 << n
    P = np.eye(dim, dtype=complex)
    for h in range(n):
        s = -1.0 if (sigma >> h) & 1 else 1.0
        P = P @ ((np.eye(dim) + s * pauli_row_matrix(int(xrows[h]), int(zrows[h]), n)) / 2.0)
    best = None
    for y in range(dim):
        col = P[:, y]
        nrm = np.linalg.norm(col)
        if nrm > 1e-9:
            best = col / nrm
            break
    if best is None:
        raise ValueError("rows stabilize no state")
    # anchor: X-pivot qubits = leading x bit of each X-block row
    xpiv = [(int(xr) & -int(xr)).bit_length() - 1 for xr in xrows if int(xr) != 0]
    support = [y for y in range(dim) if abs(best[y]) > 1e-9]
    anchor = [y for y in support if all(((y >> p) & 1) == 0 for p in xpiv)]
    if len(anchor) != 1:
        raise ValueError("anchor not unique")
    ph = best[anchor[0]] / abs(best[anchor[0]])
    return best / ph
