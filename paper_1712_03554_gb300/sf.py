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
                  "cofactor", "prob", "reduce", "amp_prep", "amplitude", "filter", "export", "reset", "segment",
                  "cond", "gprog"]
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


def _ops_consumed(ops, consumed: int) -> int:
    """Op index after `consumed` program records: a "K" right after "N"
    belongs to it, a lone "K" has no record."""
    i, r = 0, 0
    while i < len(ops) and r < consumed:
        if ops[i][0] != "K":
            r += 1
        i += 1
    while i < len(ops) and ops[i][0] == "K":
        i += 1
    return i


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
        "sf_apply_program": ([H, C.c_void_p, u64, dbl, u64, C.c_void_p, C.c_void_p], st),
        "sf_apply_program_grid": ([H, C.c_void_p, u64, dbl, C.c_void_p], st),
        "sf_run_program": ([H, C.c_void_p, u64, dbl, P64, C.POINTER(C.c_uint32), u32], st),
        "sf_set_wait_limit": ([H, u32], st),
        "sf_set_lowrank": ([H, C.c_int32], st),
        "sf_lowrank_ranks": ([H, C.POINTER(C.c_int32)], st),
        "sf_grid_program_bytes": ([H, P64], st),
        "sf_set_trace": ([H, C.c_int32], st),
        "sf_grid_program_trace": ([H, P64, u32, C.POINTER(C.c_uint32)], st),
        "sf_grid_program_plan_trace": ([H, P64, u32], st),
        "sf_apply_toffoli": ([H, u32, u32, u32], st),
        "sf_apply_cr_cofactor": ([H, u32, u32, dbl], st),
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
        "sf_campaign_create": ([u32, u32, C.c_void_p, C.POINTER(C.c_void_p)], st),
        "sf_campaign_destroy": ([H], st),
        "sf_campaign_run": ([H, C.c_void_p, C.c_void_p, u32, dbl] + [C.c_void_p] * 8, st),
        "sf_campaign_ctas": ([H], u32),
        "sf_footprint_bytes": ([u32, u64], u64),
        "sf_server_create": ([u64, u32, C.POINTER(C.c_void_p)], st),
        "sf_server_submit": ([H, C.c_void_p, C.POINTER(C.c_uint64)], st),
        "sf_server_poll": ([H, C.c_void_p, u32], u32),
        "sf_server_wait": ([H, dbl], st),
        "sf_server_stats_get": ([H, C.c_void_p], st),
        "sf_server_clock": ([H], dbl),
        "sf_server_destroy": ([H], st),
        "sf_campaign_set_shape": ([H, u32, u32], st),
        "sf_campaign_get_shape": ([H, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)], st),
        "sf_campaign_set_coalesce": ([H, u32], st),
        "sf_campaign_get_coalesce": ([H], u32),
        "sf_campaign_autotune": ([H, C.c_void_p, C.c_void_p, u32, dbl, u32, C.POINTER(C.c_float)], st),
        "sf_mf_create": ([u32, u64, u32, C.c_void_p, C.POINTER(C.c_void_p)], st),
        "sf_mf_destroy": ([H], st),
        "sf_mf_apply_clifford": ([H, C.POINTER(sf_gate), u64], st),
        "sf_mf_apply_nonclifford": ([H, u32, u32, u32, dbl, dbl], st),
        "sf_mf_apply_toffoli": ([H, u32, u32, u32, dbl], st),
        "sf_mf_apply_cr": ([H, u32, u32, dbl, dbl], st),
        "sf_mf_coalesce": ([H, dbl, C.POINTER(C.c_uint32), P64], st),
        "sf_mf_count": ([H, C.POINTER(C.c_uint32), P64], st),
        "sf_mf_amplitude": ([H, P64, PD, PD], st),
        "sf_mf_frame": ([H, u32, C.POINTER(C.c_void_p)], st),
        "sf_mf_launches": ([H], u64),
        "sf_mf_last_error": ([H], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


COALESCE_NOALLOC_MAX_ELEMS = 65536
WAIT_LIMIT_DEFAULT = 1048576
RUN_ONE_CTA = 1


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


CAMPAIGN_MAX_ELEMS = 16384
OP_DIAG, OP_MEASURE, OP_COND = 16, 32, 33
SF_OP_DTYPE = np.dtype([("kind", "<u4"), ("q0", "<u4"), ("q1", "<u4"), ("arg", "<u4"), ("param", "<f8")])


def encode_program(circuits) -> Tuple[np.ndarray, np.ndarray]:
    """sf_op records and offsets for a list of circuits in the op vocabulary of
    circuits.py: ("C", kind, q0, q1) Clifford gate; ("N", kind, q0, q1, theta)
    diagonal gate (the campaign engine always merges, so a following ("K",) is
    implied and skipped); ("M", q, u) measurement with draw u; ("Q", kind, q0,
    q1, mask) Clifford gate applied iff parity(outcomes & mask) = 1."""
    recs, offs = [], [0]
    for ops in circuits:
        for op in ops:
            t = op[0]
            if t == "C":
                recs.append((op[1], op[2], op[3], 0, 0.0))
            elif t == "N":
                recs.append((OP_DIAG + op[1], op[2], op[3], 0, float(op[4])))
            elif t == "K":
                continue
            elif t == "M":
                if op[2] is None:
                    raise ValueError("a campaign measurement needs a draw u")
                recs.append((OP_MEASURE, op[1], 0, 0, float(op[2])))
            elif t == "Q":
                mask = np.array([op[4]], dtype=np.uint64).view(np.float64)[0]
                recs.append((OP_COND, op[2], op[3], op[1], mask))
            else:
                raise ValueError(f"unknown op {op!r}")
        offs.append(len(recs))
    return np.array(recs, dtype=SF_OP_DTYPE), np.array(offs, dtype=np.uint64)


class Campaign:
    """Batched engine: many circuits of n <= 63 qubits in one persistent
    launch (sf_campaign_* in include/sf.h).  Device buffers come from torch."""

    def __init__(self, n: int, max_elems: int, stream=None):
        self.lib = load()
        self.n, self.cap = int(n), int(max_elems)
        self._stream = stream
        sh = int(stream.cuda_stream) if stream is not None else _current_stream_handle()
        self._sh = sh
        h = C.c_void_p()
        code = self.lib.sf_campaign_create(self.n, self.cap, C.c_void_p(sh), C.byref(h))
        if code != SF_OK:
            raise SFError(code, "sf_campaign_create failed")
        self.h = h

    def ctas(self) -> int:
        return int(self.lib.sf_campaign_ctas(self.h))

    def set_shape(self, threads_per_circuit: int, smem_index: bool) -> None:
        code = self.lib.sf_campaign_set_shape(self.h, int(threads_per_circuit), 1 if smem_index else 0)
        if code != SF_OK:
            raise SFError(code, "sf_campaign_set_shape failed")

    def shape(self) -> Tuple[int, bool, int]:
        """(threads per circuit, index in shared memory, CTAs)."""
        t, sm, n = C.c_uint32(), C.c_uint32(), C.c_uint32()
        self.lib.sf_campaign_get_shape(self.h, C.byref(t), C.byref(sm), C.byref(n))
        return int(t.value), bool(sm.value), int(n.value)

    def set_coalesce(self, sorted_index: bool) -> None:
        """sf_campaign_set_coalesce: merges find partners through a hash index
        (False) or the positions sorted by phase vector (True)."""
        code = self.lib.sf_campaign_set_coalesce(self.h, 1 if sorted_index else 0)
        if code != SF_OK:
            raise SFError(code, "sf_campaign_set_coalesce failed")

    def coalesce_sorted(self) -> bool:
        return bool(self.lib.sf_campaign_get_coalesce(self.h))

    def autotune(self, ops, off, nc: int, drop_eps: float = 1e-12, reps: int = 2) -> float:
        """sf_campaign_autotune on an uploaded program; returns the best ms per run."""
        ms = C.c_float()
        code = self.lib.sf_campaign_autotune(self.h, C.c_void_p(ops.data_ptr()), C.c_void_p(off.data_ptr()), nc,
                                             float(drop_eps), int(reps), C.byref(ms))
        if code != SF_OK:
            raise SFError(code, "sf_campaign_autotune failed")
        return float(ms.value)

    def upload(self, circuits):
        """Encode and copy a program to the device: (ops, offsets, n_circuits)."""
        import torch
        recs, offs = encode_program(circuits)
        if len(recs) == 0:  # the ABI wants a valid ops pointer even when every circuit is empty
            recs = np.zeros(1, dtype=SF_OP_DTYPE)
        ops = torch.from_numpy(recs.view(np.uint8).copy()).to("cuda")
        off = torch.from_numpy(offs.view(np.int64).copy()).to("cuda")
        return ops, off, len(offs) - 1

    def outputs(self, nc: int, export: bool = False):
        import torch
        dev = "cuda"
        out = {"outcomes": torch.zeros(nc, dtype=torch.int64, device=dev),
               "n_meas": torch.zeros(nc, dtype=torch.int32, device=dev),
               "k_final": torch.zeros(nc, dtype=torch.int32, device=dev),
               "norm": torch.zeros(nc, dtype=torch.float64, device=dev),
               "status": torch.zeros(nc, dtype=torch.int32, device=dev)}
        if export:
            out["sigma"] = torch.zeros(nc * self.cap, dtype=torch.int64, device=dev)
            out["amp"] = torch.zeros(nc * self.cap * 2, dtype=torch.float64, device=dev)
            out["tableau"] = torch.zeros(nc * 129, dtype=torch.int64, device=dev)
        return out

    def launch(self, ops, off, nc: int, drop_eps: float, out) -> None:
        """Asynchronous sf_campaign_run on uploaded buffers (see upload/outputs)."""
        ex = [out[k].data_ptr() if k in out else None for k in ("sigma", "amp", "tableau")]
        code = self.lib.sf_campaign_run(self.h, C.c_void_p(ops.data_ptr()), C.c_void_p(off.data_ptr()), nc,
                                        float(drop_eps), C.c_void_p(out["outcomes"].data_ptr()),
                                        C.c_void_p(out["n_meas"].data_ptr()), C.c_void_p(out["k_final"].data_ptr()),
                                        C.c_void_p(out["norm"].data_ptr()), C.c_void_p(out["status"].data_ptr()),
                                        *[C.c_void_p(p) for p in ex])
        if code != SF_OK:
            raise SFError(code, "sf_campaign_run failed")

    def run(self, circuits, drop_eps: float = 1e-12, export: bool = False):
        """Run a list of circuits; returns numpy results per circuit and, with
        export, each final frame as (x rows, z rows, r, sigma, amp) with the
        elements sorted by phase vector."""
        import torch
        ops, off, nc = self.upload(circuits)
        out = self.outputs(nc, export)
        self.launch(ops, off, nc, drop_eps, out)
        if self._stream is not None:
            self._stream.synchronize()
        else:
            torch.cuda.synchronize()
        res = {k: out[k].cpu().numpy() for k in ("outcomes", "n_meas", "k_final", "norm", "status")}
        res["outcomes"] = res["outcomes"].view(np.uint64)
        if export:
            sig = out["sigma"].cpu().numpy().view(np.uint64).reshape(nc, self.cap)
            amp = out["amp"].cpu().numpy().reshape(nc, self.cap, 2)
            tab = out["tableau"].cpu().numpy().view(np.uint64).reshape(nc, 129)
            frames = []
            for c in range(nc):
                k = int(res["k_final"][c])
                order = np.argsort(sig[c, :k], kind="stable")
                frames.append((tab[c, :self.n].copy(), tab[c, 64:64 + self.n].copy(), int(tab[c, 128]),
                               sig[c, :k][order].copy(), amp[c, :k, 0][order] + 1j * amp[c, :k, 1][order]))
            res["frames"] = frames
        return res

    def close(self):
        if getattr(self, "h", None):
            self.lib.sf_campaign_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVER_MAX_PROBES = 4


class sf_request(C.Structure):
    _fields_ = [("n_qubits", C.c_uint32), ("n_probes", C.c_uint32), ("max_elems", C.c_uint64),
                ("drop_eps", C.c_double), ("ops", C.c_void_p), ("n_ops", C.c_uint64), ("probes", C.c_void_p)]


class sf_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("n_meas", C.c_uint32), ("outcomes", C.c_uint64),
                ("k_final", C.c_uint64), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("n_probes", C.c_uint32), ("pad", C.c_uint32),
                ("amp", C.c_double * (2 * SERVER_MAX_PROBES))]


class sf_server_stats(C.Structure):
    _fields_ = [("queued", C.c_uint32), ("active", C.c_uint32), ("bytes_in_use", C.c_uint64),
                ("submitted", C.c_uint64), ("completed", C.c_uint64)]


def footprint_bytes(n: int, max_elems: int) -> int:
    return int(load().sf_footprint_bytes(int(n), int(max_elems)))


class Server:
    """Continuous-batching request loop (sf_server_* in include/sf.h): circuits
    are admitted by HBM footprint onto max_active slots, each with its own
    stream and resident frame."""

    def __init__(self, hbm_budget_bytes: int, max_active: int):
        self.lib = load()
        h = C.c_void_p()
        code = self.lib.sf_server_create(int(hbm_budget_bytes), int(max_active), C.byref(h))
        if code != SF_OK:
            raise SFError(code, "sf_server_create failed")
        self.h = h

    def submit(self, n: int, ops, max_elems: int, probes: Sequence[int] = (), drop_eps: float = 1e-12) -> int:
        """Queue one circuit (ops in the vocabulary of circuits.py, or sf_op
        records); returns its id."""
        recs = ops if isinstance(ops, np.ndarray) else encode_program([ops])[0]
        recs = np.ascontiguousarray(recs, dtype=SF_OP_DTYPE)
        W = (int(n) + 63) // 64
        pw = np.concatenate([int_to_words(int(x), W) for x in probes]) if len(probes) else np.zeros(1, np.uint64)
        req = sf_request(int(n), len(probes), int(max_elems), float(drop_eps),
                         recs.ctypes.data if len(recs) else None, len(recs), pw.ctypes.data)
        rid = C.c_uint64()
        code = self.lib.sf_server_submit(self.h, C.byref(req), C.byref(rid))
        if code != SF_OK:
            raise SFError(code, "sf_server_submit failed")
        return int(rid.value)

    def poll(self, max_results: int = 4096):
        buf = (sf_result * max_results)()
        k = self.lib.sf_server_poll(self.h, buf, max_results)
        out = []
        for r in buf[:k]:
            out.append({"id": int(r.id), "status": int(r.status), "n_meas": int(r.n_meas),
                        "outcomes": int(r.outcomes), "k_final": int(r.k_final), "t_submit": r.t_submit,
                        "t_start": r.t_start, "t_done": r.t_done,
                        "amps": [complex(r.amp[2 * p], r.amp[2 * p + 1]) for p in range(r.n_probes)]})
        return out

    def wait(self, timeout: float = -1.0) -> None:
        code = self.lib.sf_server_wait(self.h, float(timeout))
        if code != SF_OK:
            raise SFError(code, "sf_server_wait")

    def stats(self):
        st = sf_server_stats()
        self.lib.sf_server_stats_get(self.h, C.byref(st))
        return {"queued": st.queued, "active": st.active, "bytes_in_use": st.bytes_in_use,
                "submitted": st.submitted, "completed": st.completed}

    def clock(self) -> float:
        return float(self.lib.sf_server_clock(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
        if h and getattr(self, "_owned", True):
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

    def apply_toffoli_cofactor(self, c1: int, c2: int, t: int) -> None:
        """sf_apply_toffoli: TOF by cofactors (Eq. 2)."""
        self._check(self.lib.sf_apply_toffoli(self.h, int(c1), int(c2), int(t)), self.h)

    def apply_cr_cofactor(self, c: int, t: int, alpha: float) -> None:
        """sf_apply_cr_cofactor: R(alpha)_{ct} by cofactors (Eq. 3)."""
        self._check(self.lib.sf_apply_cr_cofactor(self.h, int(c), int(t), float(alpha)), self.h)

    def apply_program_device(self, dev_ops: int, n_ops: int, eps: float = 1e-12, dev_consumed: int = 0,
                             dev_meas: int = 0, max_frame: int = 0) -> None:
        """sf_apply_program on device pointers (ints; 0 for NULL)."""
        self._check(self.lib.sf_apply_program(self.h, C.c_void_p(dev_ops or None), int(n_ops), float(eps),
                                              int(max_frame), C.c_void_p(dev_consumed or None),
                                              C.c_void_p(dev_meas or None)), self.h)

    def apply_program(self, ops, eps: float = 1e-12, max_frame: int = 0):
        """Apply ops (the vocabulary of circuits.py) through sf_apply_program
        while the frame is small.  Returns (i, outcome_bits, n_meas): ops[:i]
        were applied (i counts op tuples, a coalesce after a diagonal gate
        included); continue with the per-op calls from ops[i]."""
        import torch
        recs, _ = encode_program([ops])
        if len(recs) == 0:
            return len(ops), 0, 0
        d_ops = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
        out = torch.zeros(3, dtype=torch.int64, device="cuda")
        self.apply_program_device(d_ops.data_ptr(), len(recs), eps, out.data_ptr(), out.data_ptr() + 8, max_frame)
        self.sync()
        consumed, bits, nm = (int(v) for v in out.cpu().numpy().view(np.uint64))
        return _ops_consumed(ops, consumed), bits, nm

    def apply_program_grid_device(self, dev_ops: int, n_ops: int, eps: float = 1e-12, dev_consumed: int = 0) -> None:
        """sf_apply_program_grid on device pointers (ints; 0 for NULL)."""
        self._check(self.lib.sf_apply_program_grid(self.h, C.c_void_p(dev_ops or None), int(n_ops), float(eps),
                                                   C.c_void_p(dev_consumed or None)), self.h)

    def apply_program_grid(self, ops, eps: float = 1e-12) -> int:
        """Apply ops through sf_apply_program_grid (one cooperative launch)
        up to the first measurement or conditional gate.  Returns i: ops[:i]
        were applied; continue with the per-op calls from ops[i]."""
        import torch
        recs, _ = encode_program([ops])
        if len(recs) == 0:
            return len(ops)
        d_ops = torch.from_numpy(recs.view(np.uint8).copy()).cuda()
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.apply_program_grid_device(d_ops.data_ptr(), len(recs), eps, out.data_ptr())
        self.sync()
        return _ops_consumed(ops, int(out.cpu().numpy().view(np.uint64)[0]))

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

    def run_program_records(self, recs: np.ndarray, eps: float = 1e-12, one_cta: bool = False) -> Tuple[int, int]:
        """sf_run_program on an array of sf_op records in host memory (the
        library copies them); returns (outcome bits, number of measurements).
        one_cta: SF_RUN_ONE_CTA (no whole-GPU launch)."""
        recs = np.ascontiguousarray(recs)
        bits, nm = C.c_uint64(), C.c_uint32()
        self._check(self.lib.sf_run_program(self.h, recs.ctypes.data_as(C.c_void_p), len(recs), float(eps),
                                            C.byref(bits), C.byref(nm), RUN_ONE_CTA if one_cta else 0), self.h)
        return int(bits.value), int(nm.value)

    def run_program(self, ops, eps: float = 1e-12, one_cta: bool = False) -> Tuple[int, int]:
        """The ops (circuits.py vocabulary) as one sf_run_program call."""
        recs, _ = encode_program([ops])
        return self.run_program_records(recs, eps, one_cta)

    def grid_program_bytes(self) -> int:
        """sf_grid_program_bytes: element bytes moved by the last grid program launch."""
        b = C.c_uint64()
        self._check(self.lib.sf_grid_program_bytes(self.h, C.byref(b)), self.h)
        return int(b.value)

    def set_trace(self, on: bool) -> None:
        """sf_set_trace: record per-phase times of the next grid program launches."""
        self._check(self.lib.sf_set_trace(self.h, 1 if on else 0), self.h)

    def grid_program_trace(self) -> np.ndarray:
        """sf_grid_program_trace: (phases, 13) uint64 records of the last traced launch."""
        buf = np.zeros((512, 13), dtype=np.uint64)
        n = C.c_uint32()
        self._check(self.lib.sf_grid_program_trace(self.h, buf.ctypes.data_as(C.POINTER(C.c_uint64)), 512,
                                                   C.byref(n)), self.h)
        return buf[:n.value].copy()

    def grid_program_plan_trace(self, steps: int = 64) -> np.ndarray:
        """sf_grid_program_plan_trace: (steps, 8) uint64 stamps of the planning CTAs."""
        buf = np.zeros((steps, 8), dtype=np.uint64)
        self._check(self.lib.sf_grid_program_plan_trace(self.h, buf.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                        steps), self.h)
        return buf

    def set_wait_limit(self, polls: int) -> None:
        """sf_set_wait_limit: barrier polls of the grid program before it gives up."""
        self._check(self.lib.sf_set_wait_limit(self.h, int(polls)), self.h)

    def set_lowrank(self, on: bool) -> None:
        """sf_set_lowrank: low-rank forms of the affine and cofactor maps (n > 256)."""
        self._check(self.lib.sf_set_lowrank(self.h, 1 if on else 0), self.h)

    def lowrank_ranks(self):
        """sf_lowrank_ranks: (affine, cofactor U, cofactor V) ranks, -1 = per-bit form."""
        r = (C.c_int32 * 3)()
        self._check(self.lib.sf_lowrank_ranks(self.h, r), self.h)
        return tuple(int(v) for v in r)

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


class MultiFrame:
    """A multiframe on the GPU (include/sf_multiframe.h, Sec. IV): frames with
    different stabilizer matrices whose states sum to one state."""

    def __init__(self, n: int, max_elems: int = 8192, max_frames: int = 4096, stream=None):
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
        self._check(self.lib.sf_mf_create(n, max_elems, max_frames, C.c_void_p(sh), C.byref(h)), None)
        self.h = h
        self.max_elems = max_elems

    def _check(self, code: int, h) -> None:
        if code != SF_OK:
            msg = self.lib.sf_mf_last_error(h)
            raise SFError(code, msg.decode() if msg else "")

    def close(self) -> None:
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.sf_mf_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_clifford(self, gates) -> None:
        arr = (sf_gate * len(gates))(*[sf_gate(int(g[0]), int(g[1]), int(g[2]) if len(g) > 2 else 0, 0)
                                         for g in gates])
        self._check(self.lib.sf_mf_apply_clifford(self.h, arr, len(gates)), self.h)

    def apply_nonclifford_coalesce(self, kind, q0, q1=0, theta=0.0, drop_eps=1e-12) -> None:
        self._check(self.lib.sf_mf_apply_nonclifford(self.h, kind, q0, q1, float(theta), float(drop_eps)), self.h)

    def apply_toffoli_cofactor(self, c1, c2, t, drop_eps=1e-12) -> None:
        self._check(self.lib.sf_mf_apply_toffoli(self.h, c1, c2, t, float(drop_eps)), self.h)

    def apply_cr_cofactor(self, c, t, alpha, drop_eps=1e-12) -> None:
        self._check(self.lib.sf_mf_apply_cr(self.h, c, t, float(alpha), float(drop_eps)), self.h)

    def coalesce(self, drop_eps=1e-12):
        nf, ns = C.c_uint32(), C.c_uint64()
        self._check(self.lib.sf_mf_coalesce(self.h, float(drop_eps), C.byref(nf), C.byref(ns)), self.h)
        return int(nf.value), int(ns.value)

    def count(self):
        nf, ns = C.c_uint32(), C.c_uint64()
        self._check(self.lib.sf_mf_count(self.h, C.byref(nf), C.byref(ns)), self.h)
        return int(nf.value), int(ns.value)

    def amplitude(self, x) -> complex:
        xs = np.array([int(x)], dtype=np.uint64)
        re, im = C.c_double(), C.c_double()
        self._check(self.lib.sf_mf_amplitude(self.h, xs.ctypes.data_as(C.POINTER(C.c_uint64)), C.byref(re),
                                             C.byref(im)), self.h)
        return complex(re.value, im.value)

    def frame(self, i: int) -> Frame:
        """Frame i as a borrowed Frame (valid until the next call on the multiframe)."""
        fh = C.c_void_p()
        self._check(self.lib.sf_mf_frame(self.h, i, C.byref(fh)), self.h)
        f = Frame.__new__(Frame)
        f.lib, f.n, f.h, f.W, f.max_elems, f.stream_handle = self.lib, self.n, fh, 1, self.max_elems, self.stream_handle
        f._owned = False
        return f

    def as_dict(self):
        """{(x bytes, z bytes): {sigma: amplitude}} -- the multiframe as a set."""
        out = {}
        for i in range(self.count()[0]):
            f = self.frame(i)
            x, z, _ = f.tableau()
            sig, amp = f.frame()
            out[(x.tobytes(), z.tobytes())] = {int(row[0]): complex(a) for row, a in zip(sig, amp)}
        return out

    def kernel_launches(self) -> int:
        return int(self.lib.sf_mf_launches(self.h))

