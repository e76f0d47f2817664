"""Multiframe oracle (Sec. IV, "Multiframe simulation").  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this module.  It shares no code with the CUDA library.

A multiframe is a list of frames with different stabilizer matrices that
together represent one state: Psi = sum over frames F, over elements (sigma, a)
of F, of a * psi_can(M_F, sigma).  Each frame is a FrameOracle (frame_oracle.c),
so every Clifford conjugation, global phase and cofactor below is the pinned
single-frame oracle's.

COALESCE(F), Sec. IV, followed step by step:
  * Z_k-rows: rows of the RREF matrix with no X part and a single Z literal
    (on qubit k); such a row fixes qubit k to |sigma_r>.
  * candidate pair <sigma_r, sigma_j>: equal outside the Z_k-rows, and
    a_r = i^d a_j for some d in {0,1,2,3} (tested as |a_r - i^d a_j| <= tol |a_j|
    on the canonical amplitudes).
  * Step 1 sorts the phase vectors so that candidates are next to each other:
    by their entries on the other rows, then by their entries on the Z_k-rows,
    each compared as a row vector with the first row most significant (the
    order in which the paper's worked example finds the pairs <sigma_1, sigma_2>,
    e = {2}, and <sigma_3, sigma_4>, e = {2, 3}).  The sorted list is walked
    once from the front: two neighbours that are candidates form a pair and
    are both taken; otherwise the first stays unpaired.
  * Step 2-3: the pair's differing rows e fix the qubits v_1 < ... < v_m; the
    pair member whose entry on v_1's row is 0 (qubit v_1 in |0>) is sigma_j.
    Then a_j psi_j + a_r psi_r = sqrt(2) a_j C psi_j with
    C = CNOT_{v1,v2} ... CNOT_{v1,vm} P^d_{v1} H_{v1}, so the pair becomes the
    element (sigma_j, sqrt(2) a_j) of a new frame with matrix C M C^dagger:
    the pairs sharing (e, d) form one frame, which is copied from F and
    rotated by C (ROTATE, Sec. III).  F keeps its unpaired elements.
  * Step 4 and the merge of A16: the new frames are coalesced again and frames
    with equal matrices are merged (union of elements, then Def. 1's
    coalescing of equal phase vectors), until no candidate pair is left.

Gates on a multiframe act on every frame; Toffoli and controlled-R(alpha) by
cofactors (Eq. 2, Eq. 3) are followed by the coalescing of the multiframe
(Sec. IV, gates on multiframes).  Orthogonality checks and orthogonalisation
are not part of this module.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np

from . import FrameOracle

TOL = 1e-9
_IPOW = (1, 1j, -1, -1j)
H, S, SDG, CNOT, CZ = 0, 1, 2, 6, 7  # Clifford kinds of the C ABI (sf_clifford_kind)


def zk_rows(x: np.ndarray, z: np.ndarray) -> Dict[int, int]:
    """Z_k-rows of an RREF tableau: row index -> the qubit k it stabilizes."""
    rows = {}
    for r in range(x.shape[0]):
        if np.any(x[r]):
            continue
        bits = [(w, int(v)) for w, v in enumerate(z[r]) if int(v)]
        if len(bits) == 1 and bits[0][1] & (bits[0][1] - 1) == 0:
            rows[r] = 64 * bits[0][0] + bits[0][1].bit_length() - 1
    return rows


def i_power(a_r: complex, a_j: complex, tol: float = TOL):
    """d with |a_r - i^d a_j| <= tol |a_j|, or None."""
    if abs(a_j) == 0.0:
        return None
    for d, w in enumerate(_IPOW):
        if abs(a_r - w * a_j) <= tol * abs(a_j):
            return d
    return None


def sort_key(sigma: int, zmask: int, n: int):
    rest = tuple((sigma >> r) & 1 for r in range(n) if not (zmask >> r) & 1)
    zk = tuple((sigma >> r) & 1 for r in range(n) if (zmask >> r) & 1)
    return rest, zk


def _int(ws) -> int:
    return sum(int(w) << (64 * i) for i, w in enumerate(ws))


def coalesce_frame(F: FrameOracle, tol: float = TOL) -> Tuple[List[FrameOracle], int]:
    """COALESCE(F): the frames that replace F and the number of pairs formed."""
    n = F.n
    x, z, _ = F.tableau()
    sig, amp = F.frame()
    zr = zk_rows(x, z)
    zmask = sum(1 << r for r in zr)
    s = [_int(row) for row in sig]
    k = len(s)
    order = sorted(range(k), key=lambda j: sort_key(s[j], zmask, n))
    paired = [False] * k
    classes: Dict[Tuple[int, int], List[int]] = {}
    i = 0
    while i + 1 < k:
        a, b = order[i], order[i + 1]
        e = s[a] ^ s[b]
        if e and not (e & ~zmask):
            v1row = min((r for r in zr if (e >> r) & 1), key=lambda r: zr[r])
            j, r_ = (a, b) if not (s[a] >> v1row) & 1 else (b, a)
            d = i_power(amp[r_], amp[j], tol)
            if d is not None:
                classes.setdefault((e, d), []).append(j)
                paired[a] = paired[b] = True
                i += 2
                continue
        i += 1
    if not classes:
        return [F], 0
    out = []
    rest = [j for j in range(k) if not paired[j]]
    if rest:
        G = FrameOracle(n)
        G.set_state(x, z, sig[rest], amp[rest])
        out.append(G)
    for (e, d), owners in sorted(classes.items()):
        V = sorted(zr[r] for r in zr if (e >> r) & 1)
        G = FrameOracle(n)
        G.set_state(x, z, sig[owners], amp[owners] * math.sqrt(2.0))
        G.apply_clifford([(H, V[0], 0)] + [(S, V[0], 0)] * d + [(CNOT, V[0], v) for v in V[1:]])
        out.append(G)
    return out, sum(len(o) for o in classes.values())


def canonical_circuit(x: np.ndarray, z: np.ndarray, n: int) -> List[Tuple[int, int, int]]:
    """A stabilizer circuit C with C M C^dagger made of Z_k-rows (Sec. IV,
    extended coalescing, via Corollary 1's computational-basis form).  Signs
    are ignored: only the unsigned group matters for the rows' form.  Steps:
    Gauss-Jordan on the X part (row operations leave the group unchanged);
    CNOT(p_i, j) clears the X bit of row i at each non-pivot column j; the
    X-free rows, reduced, are single Z literals off the X pivots and clear the
    X rows' Z bits there; S on p_i clears a Y, CZ(p_i, p_k) clears the
    symmetric pair of Z bits between two X rows; H on every X pivot."""
    X = np.array([[(int(x[r][q >> 6]) >> (q & 63)) & 1 for q in range(n)] for r in range(n)], dtype=bool)
    Z = np.array([[(int(z[r][q >> 6]) >> (q & 63)) & 1 for q in range(n)] for r in range(n)], dtype=bool)
    gates: List[Tuple[int, int, int]] = []

    def conj(kind, a, b=0):
        gates.append((kind, a, b))
        if kind == H:
            X[:, a], Z[:, a] = Z[:, a].copy(), X[:, a].copy()
        elif kind == S:
            Z[:, a] ^= X[:, a]
        elif kind == CNOT:
            X[:, b] ^= X[:, a]
            Z[:, a] ^= Z[:, b]
        else:  # CZ
            Z[:, b] ^= X[:, a]
            Z[:, a] ^= X[:, b]

    def reduce(P, first):
        """Gauss-Jordan of plane P with pivot rows taken from rows first.. and
        every other row reduced; returns the pivot columns."""
        piv, r = [], first
        for col in range(n):
            rows = [i for i in range(r, n) if P[i, col]]
            if not rows:
                continue
            i0 = rows[0]
            X[[r, i0]] = X[[i0, r]]
            Z[[r, i0]] = Z[[i0, r]]
            for i in range(n):
                if i != r and P[i, col]:
                    X[i] ^= X[r]
                    Z[i] ^= Z[r]
            piv.append(col)
            r += 1
        return piv

    piv = reduce(X, 0)
    rx = len(piv)
    for i, p in enumerate(piv):
        for j in range(n):
            if j not in piv and X[i, j]:
                conj(CNOT, p, j)
    reduce(Z, rx)  # the X-free rows: single Z literals off the X pivots
    for i, p in enumerate(piv):
        if Z[i, p]:
            conj(S, p)
    for i in range(rx):
        for k in range(i + 1, rx):
            if Z[i, piv[k]]:
                conj(CZ, piv[i], piv[k])
    for p in piv:
        conj(H, p)
    assert not X.any() and all(Z[i].sum() == 1 for i in range(n))
    return gates


def coalesce_frame_extended(F: FrameOracle, tol: float = TOL) -> Tuple[List[FrameOracle], int]:
    """Extended COALESCE (Sec. IV): ROTATE F by a circuit C that maps M to
    computational-basis form (every row a Z_k-row), COALESCE, and ROTATE every
    frame produced back by C^dagger."""
    n = F.n
    x, z, _ = F.tableau()
    C = canonical_circuit(x, z, n)
    sig, amp = F.frame()
    G = FrameOracle(n)
    G.set_state(x, z, sig, amp)
    if C:
        G.apply_clifford(C)
    out, pairs = coalesce_frame(G, tol)
    Cinv = [(SDG if k == S else k, a, b) for (k, a, b) in reversed(C)]
    if Cinv:
        for o in out:
            o.apply_clifford(Cinv)
    return out, pairs


def merge_frames(frames: List[FrameOracle], eps: float = 1e-12) -> List[FrameOracle]:
    """A16: frames with equal stabilizer matrices become one frame (the union
    of their elements, then Def. 1 coalescing).  Empty frames are dropped."""
    groups: Dict[bytes, List[FrameOracle]] = {}
    for F in frames:
        x, z, _ = F.tableau()
        groups.setdefault(x.tobytes() + z.tobytes(), []).append(F)
    out = []
    for fs in groups.values():
        if len(fs) == 1:
            if fs[0].size():
                out.append(fs[0])
            continue
        x, z, _ = fs[0].tableau()
        parts = [F.frame() for F in fs]
        G = FrameOracle(fs[0].n)
        G.set_state(x, z, np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
        G.coalesce(eps)
        if G.size():
            out.append(G)
    return out


class MultiFrameOracle:
    """A list of FrameOracle frames representing one state (Sec. IV)."""

    def __init__(self, n: int, tol: float = TOL, eps: float = 1e-12, reading: str = "printed"):
        """reading: "printed" (COALESCE on the Z_k-rows of the frame's own
        matrix, the GPU library's reading) or "extended" (each frame first
        rotated to computational-basis form)."""
        if reading not in ("printed", "extended"):
            raise ValueError(reading)
        self.reading = reading
        self.n = n
        self.W = (n + 63) // 64
        self.tol = tol
        self.eps = eps
        self.frames: List[FrameOracle] = [FrameOracle(n)]

    def apply_clifford(self, gates):
        for F in self.frames:
            F.apply_clifford(gates)

    def apply_nonclifford_coalesce(self, kind, q0, q1=0, theta=0.0):
        for F in self.frames:
            F.apply_nonclifford(kind, q0, q1, theta)
            F.coalesce(self.eps)
        self.frames = [F for F in self.frames if F.size()]

    def apply_toffoli_cofactor(self, c1, c2, t):
        for F in self.frames:
            F.apply_toffoli_cofactor(c1, c2, t)
            F.coalesce(self.eps)
        return self.coalesce()

    def apply_cr_cofactor(self, c, t, alpha):
        for F in self.frames:
            F.apply_cr_cofactor(c, t, alpha)
            F.coalesce(self.eps)
        return self.coalesce()

    def coalesce(self):
        """Merge, then COALESCE every frame and merge again until no candidate
        pair is left.  Returns (frames, states)."""
        frames = merge_frames(self.frames, self.eps)
        while True:
            new, pairs = [], 0
            step = coalesce_frame_extended if self.reading == "extended" else coalesce_frame
            for F in frames:
                out, p = step(F, self.tol)
                new += out
                pairs += p
            frames = merge_frames(new, self.eps)
            if not pairs:
                break
        self.frames = frames
        return self.count()

    def count(self):
        return len(self.frames), sum(F.size() for F in self.frames)

    def amplitude(self, y: int) -> complex:
        return sum(F.amplitude(y) for F in self.frames)

    def as_dict(self):
        """{(x bytes, z bytes): {sigma: amplitude}} -- the multiframe as a set."""
        out = {}
        for F in self.frames:
            x, z, _ = F.tableau()
            sig, amp = F.frame()
            out[(x.tobytes(), z.tobytes())] = {_int(row): complex(a) for row, a in zip(sig, amp)}
        return out
