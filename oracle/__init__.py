"""CPU oracles for the stabilizer-frame hot path.  TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The CUDA library never imports, links or calls it, and it shares
no code with the CUDA library.

  FrameOracle  -- plain C stabilizer-frame simulator (frame_oracle.c), the
                  paper's algorithm step by step: Table 1/Table 2 lookups,
                  Gauss-Jordan RREF after every gate (Invariant 1), the
                  five-step global-phase rule of Sec. III per element, branching
                  of diagonal non-Clifford gates, COFACTOR for measurement.
                  set_threads(t) splits its per-element loops into t ranges
                  run by t threads (Sec. V); the default is sequential.
  DenseOracle  -- numpy state vector (the "array of complex amplitudes"
                  check the paper uses in Sec. VI), n <= 22.
  multiframe   -- MultiFrameOracle: lists of FrameOracle frames, COALESCE into
                  new frames and the merge of equal matrices (Sec. IV).

Pins (tests/test_oracle_*.py) tie them to Tables 1 and 2, the paper's worked
examples (Ex. 1, Ex. 2, the P|1> = i|1> example of Sec. II-B, the COALESCE
example of Sec. IV), closed forms (QFT, GHZ, Cuccaro addition) and brute force
over every phase vector at n <= 6.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .dense import DenseOracle  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frame_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile frame_oracle.c with gcc (portable flags: x86_64 and aarch64)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm",
                                   "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, u32, u64p, dp, szp = C.c_void_p, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_size_t)
        lib.of_create.restype = vp
        lib.of_create.argtypes = [C.c_int]
        lib.of_destroy.argtypes = [vp]
        lib.of_reset.argtypes = [vp]
        lib.of_clifford.argtypes = [vp, C.POINTER(C.c_uint32), C.c_size_t]
        lib.of_nonclifford.argtypes = [vp, u32, u32, u32, C.c_double]
        lib.of_coalesce.argtypes = [vp, C.c_double, szp]
        lib.of_measure.argtypes = [vp, u32, C.c_int, dp, dp]
        lib.of_toffoli_cofactor.argtypes = [vp, u32, u32, u32]
        lib.of_cr_cofactor.argtypes = [vp, u32, u32, C.c_double]
        lib.of_amplitude.argtypes = [vp, u64p, dp, dp]
        lib.of_get_tableau.argtypes = [vp, u64p, u64p, C.POINTER(C.c_uint32)]
        lib.of_get_frame.argtypes = [vp, u64p, dp, C.c_size_t, szp]
        lib.of_size.restype = C.c_size_t
        lib.of_size.argtypes = [vp]
        lib.of_set_state.argtypes = [vp, u64p, u64p, u64p, dp, C.c_size_t]
        lib.of_basis_amp.argtypes = [vp, u64p, u64p, dp, dp]
        lib.of_is_rref.argtypes = [vp]
        lib.of_set_threads.restype = C.c_int
        lib.of_set_threads.argtypes = [C.c_int]
        lib.ot_pauli_mult.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
        lib.ot_conjugate.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        _lib = lib
    return _lib


def _u64(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _f64(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def int_to_words(v: int, W: int) -> np.ndarray:
    return np.array([(v >> (64 * w)) & ((1 << 64) - 1) for w in range(W)], dtype=np.uint64)


def words_to_int(ws) -> int:
    return sum(int(w) << (64 * i) for i, w in enumerate(ws))


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


class FrameOracle:
    """Plain CPU stabilizer frame (see frame_oracle.c)."""

    def __init__(self, n: int):
        self.lib = _load()
        self.n = n
        self.W = (n + 63) // 64
        self.h = self.lib.of_create(n)
        if not self.h:
            raise OracleError(1, "create")

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.of_destroy(h)

    def _chk(self, st, what):
        if st:
            raise OracleError(st, what)

    def reset(self):
        self.lib.of_reset(self.h)

    def apply_clifford(self, gates):
        arr = np.zeros((len(gates), 4), dtype=np.uint32)
        for i, g in enumerate(gates):
            arr[i, :3] = g[:3]
        self._chk(self.lib.of_clifford(self.h, arr.ctypes.data_as(C.POINTER(C.c_uint32)), len(gates)), "clifford")

    def apply_nonclifford(self, kind, q0, q1=0, theta=0.0):
        self._chk(self.lib.of_nonclifford(self.h, kind, q0, q1, float(theta)), "nonclifford")

    def coalesce(self, eps=1e-12):
        k = C.c_size_t()
        self._chk(self.lib.of_coalesce(self.h, float(eps), C.byref(k)), "coalesce")
        return k.value

    def apply_toffoli_cofactor(self, c1, c2, t):
        """TOF by cofactors (Eq. 2)."""
        self._chk(self.lib.of_toffoli_cofactor(self.h, c1, c2, t), "toffoli")

    def apply_cr_cofactor(self, c, t, alpha):
        """R(alpha)_{ct} by cofactors (Eq. 3)."""
        self._chk(self.lib.of_cr_cofactor(self.h, c, t, float(alpha)), "cr")

    def measure(self, q, collapse=-1):
        p0, p1 = C.c_double(), C.c_double()
        self._chk(self.lib.of_measure(self.h, q, collapse, C.byref(p0), C.byref(p1)), "measure")
        return p0.value, p1.value

    def amplitude(self, x: int) -> complex:
        xs = int_to_words(x, self.W)
        re, im = C.c_double(), C.c_double()
        self._chk(self.lib.of_amplitude(self.h, _u64(xs), C.byref(re), C.byref(im)), "amplitude")
        return complex(re.value, im.value)

    def size(self) -> int:
        return int(self.lib.of_size(self.h))

    def tableau(self):
        x = np.zeros((self.n, self.W), dtype=np.uint64)
        z = np.zeros((self.n, self.W), dtype=np.uint64)
        r = C.c_uint32()
        self._chk(self.lib.of_get_tableau(self.h, _u64(x), _u64(z), C.byref(r)), "tableau")
        return x, z, r.value

    def frame(self):
        k0 = self.size()
        sig = np.zeros((max(k0, 1), self.W), dtype=np.uint64)
        amp = np.zeros((max(k0, 1), 2), dtype=np.float64)
        k = C.c_size_t()
        self._chk(self.lib.of_get_frame(self.h, _u64(sig), _f64(amp), max(k0, 1), C.byref(k)), "frame")
        k = k.value
        return sig[:k].copy(), amp[:k, 0] + 1j * amp[:k, 1]

    def set_state(self, x, z, sig, amps):
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
        sig = np.ascontiguousarray(np.asarray(sig, dtype=np.uint64).reshape(-1, self.W))
        a = np.ascontiguousarray(np.stack([np.real(amps), np.imag(amps)], axis=-1).astype(np.float64))
        self._chk(self.lib.of_set_state(self.h, _u64(x), _u64(z), _u64(sig), _f64(a), len(sig)), "set_state")

    def basis_amp(self, sigma: int, y: int) -> complex:
        s = int_to_words(sigma, self.W)
        yy = int_to_words(y, self.W)
        re, im = C.c_double(), C.c_double()
        self.lib.of_basis_amp(self.h, _u64(s), _u64(yy), C.byref(re), C.byref(im))
        return complex(re.value, im.value)

    def is_rref(self) -> bool:
        return bool(self.lib.of_is_rref(self.h))


def set_threads(t: int) -> int:
    """Number of element ranges (threads) the per-element loops of every
    FrameOracle are split into (Sec. V); 1, the default, runs them
    sequentially.  Returns the value in effect."""
    return int(_load().of_set_threads(int(t)))


def pauli_mult(a: int, b: int):
    """Table 1 lookup: literal a * literal b -> (i-power, literal)."""
    ph = C.c_int()
    res = _load().ot_pauli_mult(a, b, C.byref(ph))
    return ph.value, res


def conjugate(kind: int, l0: int, l1: int = 0):
    """Table 2 conjugation of a literal pair -> (sign bit, l0', l1')."""
    a, b = C.c_int(l0), C.c_int(l1)
    s = _load().ot_conjugate(kind, C.byref(a), C.byref(b))
    return s, a.value, b.value
