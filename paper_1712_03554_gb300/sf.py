"""Python binding of libsf (include/sf.h): argument marshalling only.

Every operation runs in the CUDA library; this module converts Python values to
the C ABI and back.  If libsf.so cannot be built or loaded the constructor
raises: there is no CPU fallback.  PyTorch, when present, supplies the CUDA
stream (torch.cuda.current_stream()).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

from . import _build

SF_OK, SF_EINVAL, SF_ENOMEM, SF_ECAPACITY, SF_ECUDA, SF_ETIMEOUT, SF_ESTATE, SF_EINTERNAL = range(8)
# kernel classes (SF_K_* in include/sf.h)
KERNEL_CLASSES = ["clifford", "affine", "branch", "branch_merge", "insert", "compact", "index", "measure_prep",
                  "cofactor", "prob", "reduce", "amp_prep", "amplitude", "filter", "export", "reset"]
STATUS_NAMES = {0: "SF_OK", 1: "SF_EINVAL", 2: "SF_ENOMEM", 3: "SF_ECAPACITY", 4: "SF_ECUDA",
                5: "SF_ETIMEOUT", 6: "SF_ESTATE", 7: "SF_EINTERNAL"}

_lib = None


class SFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class sf_gate(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("q0", C.c_uint32), ("q1", C.c_uint32), ("pad", C.c_uint32)]


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> C.CDLL:
    """Load libsf.so (building it first if needed).  Raises when unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise SFError(SF_ECUDA, f"libsf.so not found at {path}")
    lib = C.CDLL(path)
    H, st, u32, u64, dbl = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double
    P64, PD = C.POINTER(C.c_uint64), C.POINTER(C.c_double)
    sig = {
        "sf_create": ([u32, u64, C.c_void_p, C.POINTER(C.c_void_p)], st),
        "sf_destroy": ([H], st),
        "sf_reset": ([H], st),
        "sf_apply_clifford": ([H, C.POINTER(sf_gate), u64], st),
        "sf_apply_clifford_device": ([H, C.c_void_p, u64], st),
        "sf_apply_nonclifford": ([H, u32, u32, u32, dbl], st),
        "sf_apply_nonclifford_coalesce": ([H, u32, u32, u32, dbl, dbl], st),
        "sf_coalesce": ([H, dbl, P64], st),
        "sf_measure": ([H, u32, C.c_int32, PD, PD], st),
        "sf_amplitude": ([H, P64, PD, PD], st),
        "sf_size": ([H, P64], st),
        "sf_sync": ([H], st),
        "sf_get_tableau": ([H, P64, P64, C.POINTER(C.c_uint32)], st),
        "sf_get_frame": ([H, P64, PD, u64, P64], st),
        "sf_words": ([H], u32),
        "sf_kernel_launches": ([H], u64),
        "sf_host_state": ([H], u32),
        "sf_set_host_state": ([H, u32], st),
        "sf_get_internal": ([H, P64, P64, C.POINTER(C.c_uint32), PD], st),
        "sf_time_kernel": ([H, C.c_int32], st),
        "sf_kernel_time": ([H, PD, P64], st),
        "sf_last_error": ([H], C.c_char_p),
        "sf_coalesce_noalloc": ([C.c_void_p, C.c_void_p, u64, u32, dbl, C.c_void_p, C.c_void_p, P64, C.c_void_p],
                                st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


COALESCE_NOALLOC_MAX_ELEMS = 65536


def coalesce_noalloc(sigma_in: int, amp_in: int, k_in: int, n_words: int, drop_eps: float, sigma_out: int,
                     amp_out: int, stream: int = 0) -> int:
    """sf_coalesce_noalloc on device pointers (ints); returns the output count.
    For callers that cannot allocate device memory (see include/sf.h)."""
    lib = load()
    k = C.c_uint64()
    code = lib.sf_coalesce_noalloc(C.c_void_p(sigma_in), C.c_void_p(amp_in), k_in, n_words, float(drop_eps),
                                   C.c_void_p(sigma_out), C.c_void_p(amp_out), C.byref(k), C.c_void_p(stream))
    if code != SF_OK:
        raise SFError(code, "sf_coalesce_noalloc failed")
    return int(k.value)


def _current_stream_handle() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def int_to_words(v: int, W: int) -> np.ndarray:
    return np.array([(v >> (64 * w)) & ((1 << 64) - 1) for w in range(W)], dtype=np.uint64)


class Frame:
    """One stabilizer frame resident on the GPU (see include/sf.h)."""

    def __init__(self, n: int, max_elems: int, stream=None):
        self.lib = load()
        self.n = n
        if stream is None:
            sh = _current_stream_handle()
        elif isinstance(stream, int):
            sh = stream
        else:
            sh = int(stream.cuda_stream)
        self.stream_handle = sh
        h = C.c_void_p()
        self._check(self.lib.sf_create(n, max_elems, C.c_void_p(sh), C.byref(h)), None)
        self.h = h
        self.W = int(self.lib.sf_words(self.h))
        self.max_elems = max_elems

    # -- plumbing
    def _check(self, code: int, h) -> None:
        if code != SF_OK:
            msg = self.lib.sf_last_error(h)
            raise SFError(code, msg.decode() if msg else "")

    def close(self) -> None:
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.sf_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the calls of include/sf.h
    def reset(self) -> None:
        self._check(self.lib.sf_reset(self.h), self.h)

    def apply_clifford(self, gates: Sequence[Tuple[int, int, int]]) -> None:
        arr = (sf_gate * len(gates))()
        for i, g in enumerate(gates):
            arr[i].kind, arr[i].q0, arr[i].q1 = int(g[0]), int(g[1]), int(g[2])
        self._check(self.lib.sf_apply_clifford(self.h, arr, len(gates)), self.h)

    def apply_clifford_device(self, dev_ptr: int, n_gates: int) -> None:
        self._check(self.lib.sf_apply_clifford_device(self.h, C.c_void_p(dev_ptr), n_gates), self.h)

    def apply_nonclifford(self, kind: int, q0: int, q1: int = 0, theta: float = 0.0) -> None:
        self._check(self.lib.sf_apply_nonclifford(self.h, kind, q0, q1, float(theta)), self.h)

    def apply_nonclifford_coalesce(self, kind: int, q0: int, q1: int = 0, theta: float = 0.0,
                                   eps: float = 1e-12) -> None:
        self._check(self.lib.sf_apply_nonclifford_coalesce(self.h, kind, q0, q1, float(theta), float(eps)), self.h)

    def coalesce(self, eps: float = 1e-12, sync: bool = False) -> Optional[int]:
        if sync:
            k = C.c_uint64()
            self._check(self.lib.sf_coalesce(self.h, float(eps), C.byref(k)), self.h)
            return int(k.value)
        self._check(self.lib.sf_coalesce(self.h, float(eps), None), self.h)
        return None

    def measure(self, q: int, collapse: int = -1) -> Tuple[float, float]:
        p0, p1 = C.c_double(), C.c_double()
        self._check(self.lib.sf_measure(self.h, q, collapse, C.byref(p0), C.byref(p1)), self.h)
        return p0.value, p1.value

    def amplitude(self, x) -> complex:
        xs = int_to_words(int(x), self.W) if not isinstance(x, np.ndarray) else np.ascontiguousarray(x, np.uint64)
        re, im = C.c_double(), C.c_double()
        self._check(self.lib.sf_amplitude(self.h, xs.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(re),
                                          C.byref(im)), self.h)
        return complex(re.value, im.value)

    def size(self) -> int:
        k = C.c_uint64()
        self._check(self.lib.sf_size(self.h, C.byref(k)), self.h)
        return int(k.value)

    def sync(self) -> None:
        self._check(self.lib.sf_sync(self.h), self.h)

    def internal(self):
        """(dx, dz, de, g): destabilizer rows and global phase of the device state."""
        dx = np.zeros((self.n, self.W), dtype=np.uint64)
        dz = np.zeros((self.n, self.W), dtype=np.uint64)
        de = np.zeros(self.n, dtype=np.uint32)
        g = np.zeros(2, dtype=np.float64)
        P = C.POINTER(C.c_uint64)
        self._check(self.lib.sf_get_internal(self.h, dx.ctypes.data_as(P), dz.ctypes.data_as(P),
                                             de.ctypes.data_as(C.POINTER(C.c_uint32)),
                                             g.ctypes.data_as(C.POINTER(C.c_double))), self.h)
        return dx, dz, de, complex(g[0], g[1])

    def host_state(self) -> int:
        """Token of the host-side bookkeeping (restore it after replaying a graph)."""
        return int(self.lib.sf_host_state(self.h))

    def set_host_state(self, token: int) -> None:
        self._check(self.lib.sf_set_host_state(self.h, token), self.h)

    def kernel_launches(self) -> int:
        return int(self.lib.sf_kernel_launches(self.h))

    def time_kernel(self, kernel_class) -> None:
        kid = KERNEL_CLASSES.index(kernel_class) if isinstance(kernel_class, str) else int(kernel_class)
        self._check(self.lib.sf_time_kernel(self.h, kid), self.h)

    def kernel_time(self) -> Tuple[float, int]:
        ms, cnt = C.c_double(), C.c_uint64()
        self._check(self.lib.sf_kernel_time(self.h, C.byref(ms), C.byref(cnt)), self.h)
        return float(ms.value), int(cnt.value)

    def tableau(self):
        x = np.zeros((self.n, self.W), dtype=np.uint64)
        z = np.zeros((self.n, self.W), dtype=np.uint64)
        r = C.c_uint32()
        P = C.POINTER(C.c_uint64)
        self._check(self.lib.sf_get_tableau(self.h, x.ctypes.data_as(P), z.ctypes.data_as(P), C.byref(r)), self.h)
        return x, z, int(r.value)

    def frame(self):
        k0 = self.size()
        cap = max(k0, 1)
        sig = np.zeros((cap, self.W), dtype=np.uint64)
        amp = np.zeros((cap, 2), dtype=np.float64)
        k = C.c_uint64()
        self._check(self.lib.sf_get_frame(self.h, sig.ctypes.data_as(C.POINTER(C.c_uint64)),
                                          amp.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(k)), self.h)
        k = int(k.value)
        return sig[:k].copy(), amp[:k, 0] + 1j * amp[:k, 1]
