"""Thin ctypes binding of libqk (include/qk.h) -- argument marshalling only.

Every operation on amplitudes runs in libqk's CUDA kernels.  If the shared
library has not been built, importing this module raises: there is no CPU
fallback.  Build it with ``python -m paper_1908_07187_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqk.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libqk.so is not built ({LIB_PATH}); run python -m paper_1908_07187_gb300.build")

_lib = ctypes.CDLL(LIB_PATH)

QK_OK, QK_EINVAL, QK_ENOMEM, QK_EBUDGET, QK_ENOTBIJECTIVE, QK_ENOTUNITARY, QK_ECUDA, QK_ETIMEOUT, QK_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
QK_C64, QK_C128 = 0, 1
QK_EXEC_PLAIN, QK_EXEC_FUSED = 0, 1
NUM_LAUNCH_CLASSES = 7
LAUNCH_CLASSES = ("tile", "u2", "phase", "block", "perm", "measure", "other")

GATE = {
    "x": -1, "y": -2, "z": -3, "h": -4, "s": -5, "sdg": -6, "t": -7, "tdg": -8,
    "u3": -9, "p": -10, "rz": -11, "swap": -12,
}


# qk_gate_op (include/qk.h): one entry of a batch gate list, C layout
GATE_OP_DTYPE = np.dtype([("gate_id", np.int32), ("target", np.int32), ("nc", np.int32), ("ncc", np.int32),
                          ("np", np.int32), ("controls", np.int32, 4), ("cond", np.int32, 4),
                          ("params", np.float64, 3)], align=True)
assert GATE_OP_DTYPE.itemsize == 80


def layer_gate_ops(n: int, depth: int, angles) -> np.ndarray:
    """The gate list of a U3 + CZ layer circuit as qk_gate_op entries (marshalling
    only): layer L is U3(angles[L, q]) on every qubit q, then CZ on the pairs
    (q, q+1) with q = L mod 2, L mod 2 + 2, ..."""
    angles = np.asarray(angles, dtype=np.float64).reshape(depth, n, 3)
    per = [n + len(range(L % 2, n - 1, 2)) for L in range(depth)]
    out = np.zeros(sum(per), dtype=GATE_OP_DTYPE)
    pos = 0
    for L in range(depth):
        u = out[pos:pos + n]
        u["gate_id"] = GATE["u3"]
        u["target"] = np.arange(n)
        u["np"] = 3
        u["params"] = angles[L]
        pos += n
        qs = np.arange(L % 2, n - 1, 2)
        z = out[pos:pos + len(qs)]
        z["gate_id"] = GATE["z"]
        z["target"] = qs + 1
        z["nc"] = 1
        z["controls"][:, 0] = qs
        pos += len(qs)
    return out


class Options(ctypes.Structure):
    _fields_ = [("exec_mode", ctypes.c_int), ("tile_qubits", ctypes.c_int), ("max_pending", ctypes.c_int),
                ("profile", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
                ("no_tensor_cores", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


_P = ctypes.c_void_p
_IP = ctypes.POINTER(ctypes.c_int)
_DP = ctypes.POINTER(ctypes.c_double)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_U8P = ctypes.POINTER(ctypes.c_uint8)

_SIGS = {
    "qk_create": ([ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.POINTER(Options)], ctypes.c_int),
    "qk_destroy": ([_P], ctypes.c_int),
    "qk_add_qubits": ([_P, ctypes.c_int, _IP], ctypes.c_int),
    "qk_add_cbits": ([_P, ctypes.c_int, _IP], ctypes.c_int),
    "qk_define_gate_matrix": ([_P, ctypes.c_int, _DP, ctypes.c_double, _IP], ctypes.c_int),
    "qk_define_gate_perm_mulmod": ([_P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _IP], ctypes.c_int),
    "qk_define_gate_perm_table": ([_P, ctypes.c_int, _U64P, _IP], ctypes.c_int),
    "qk_apply_perm_mulmod_noalloc": ([_P, ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint64, _P], ctypes.c_int),
    "qk_apply_gate": ([_P, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int, _DP,
                       ctypes.c_int], ctypes.c_int),
    "qk_apply_rphase_cbits": ([_P, ctypes.c_int, _IP, ctypes.c_int], ctypes.c_int),
    "qk_apply_kitaev_stage": ([_P, ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int], ctypes.c_int),
    "qk_measure": ([_P, _IP, ctypes.c_int, _DP, _IP, _U64P], ctypes.c_int),
    "qk_read_cbits": ([_P, _U8P, ctypes.c_int], ctypes.c_int),
    "qk_write_cbits": ([_P, ctypes.c_int, _U8P, ctypes.c_int], ctypes.c_int),
    "qk_get_state": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "qk_set_state": ([_P, _P, ctypes.c_size_t], ctypes.c_int),
    "qk_reset": ([_P], ctypes.c_int),
    "qk_device_state": ([_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "qk_flush": ([_P], ctypes.c_int),
    "qk_sync": ([_P], ctypes.c_int),
    "qk_selftest_timeout": ([_P], ctypes.c_int),
    "qk_num_qubits": ([_P], ctypes.c_int),
    "qk_num_cbits": ([_P], ctypes.c_int),
    "qk_get_counters": ([_P, _U64P, _U64P, _U64P], ctypes.c_int),
    "qk_reset_counters": ([_P], ctypes.c_int),
    "qk_profile": ([_P, _U64P, _DP, _DP], ctypes.c_int),
    "qk_capture_begin": ([_P], ctypes.c_int),
    "qk_capture_end": ([_P, ctypes.POINTER(_P)], ctypes.c_int),
    "qk_graph_launch": ([_P], ctypes.c_int),
    "qk_graph_destroy": ([_P], ctypes.c_int),
    "qk_batch_create": ([ctypes.POINTER(_P), _P], ctypes.c_int),
    "qk_batch_destroy": ([_P], ctypes.c_int),
    "qk_batch_clear": ([_P], ctypes.c_int),
    "qk_batch_add_circuit": ([_P, ctypes.c_int, ctypes.c_int, _IP], ctypes.c_int),
    "qk_batch_apply_gate": ([_P, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int, _IP, ctypes.c_int, _DP,
                             ctypes.c_int], ctypes.c_int),
    "qk_batch_apply_mulmod": ([_P, _IP, ctypes.c_int, _IP, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64],
                              ctypes.c_int),
    "qk_batch_apply_gates": ([_P, _P, ctypes.c_int], ctypes.c_int),
    "qk_batch_measure": ([_P, _IP, ctypes.c_int, _DP, _IP], ctypes.c_int),
    "qk_batch_run": ([_P, ctypes.c_int], ctypes.c_int),
    "qk_batch_done": ([_P], ctypes.c_int),
    "qk_batch_read": ([_P, ctypes.c_int, _U8P, ctypes.c_int, _P, ctypes.c_size_t], ctypes.c_int),
    "qk_batch_read_all_cbits": ([_P, _U8P, ctypes.c_size_t], ctypes.c_int),
    "qk_batch_num_circuits": ([_P], ctypes.c_int),
    "qk_batch_stats": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "qk_apply_gates": ([_P, _P, ctypes.c_int], ctypes.c_int),
    "qk_apply_modexp": ([_P, _IP, ctypes.c_int, _IP, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_uint64,
                         _IP, ctypes.c_int], ctypes.c_int),
    "qk_batch_last_error": ([_P], ctypes.c_char_p),
    "qk_last_error": ([_P], ctypes.c_char_p),
    "qk_status_str": ([ctypes.c_int], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def exported_symbols():
    """Names of the C entry points this binding uses (all declared in include/qk.h)."""
    return list(_SIGS)


class QKError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.qk_status_str(status).decode()}: {msg}")
        self.status = status


def _ints(xs: Optional[Sequence[int]]):
    xs = list(xs or [])
    return (ctypes.c_int * max(1, len(xs)))(*xs), len(xs)


class Context:
    """One libqk context: a state vector on the current CUDA device."""

    def __init__(self, precision: str = "c64", exec_mode: str = "fused", stream: Optional[int] = None,
                 tile_qubits: int = 0, profile: bool = False, hbm_budget_bytes: int = 0, max_pending: int = 0,
                 tensor_cores: bool = True):
        opt = Options()
        opt.exec_mode = QK_EXEC_FUSED if exec_mode == "fused" else QK_EXEC_PLAIN
        if exec_mode not in ("fused", "plain"):
            raise ValueError("exec_mode must be 'fused' or 'plain'")
        opt.tile_qubits = tile_qubits
        opt.max_pending = max_pending
        opt.profile = 1 if profile else 0
        opt.hbm_budget_bytes = hbm_budget_bytes
        opt.no_tensor_cores = 0 if tensor_cores else 1
        self.precision = precision
        self.cdtype = np.complex64 if precision == "c64" else np.complex128
        prec = QK_C64 if precision == "c64" else QK_C128
        if precision not in ("c64", "c128"):
            raise ValueError("precision must be 'c64' or 'c128'")
        h = _P()
        st = _lib.qk_create(ctypes.byref(h), prec, _P(stream) if stream else None, ctypes.byref(opt))
        if st != QK_OK:
            raise QKError(st, "qk_create failed")
        self._h = h
        self._perm_cache: Dict[Tuple, int] = {}
        self._mat_cache: Dict[bytes, int] = {}

    # -- plumbing -------------------------------------------------------------
    def _check(self, st: int):
        if st != QK_OK:
            raise QKError(st, _lib.qk_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.qk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_qubits(self) -> int:
        return _lib.qk_num_qubits(self._h)

    @property
    def n_cbits(self) -> int:
        return _lib.qk_num_cbits(self._h)

    # -- the paper's commands ------------------------------------------------------
    def add_qubits(self, n: int) -> int:
        first = ctypes.c_int(0)
        self._check(_lib.qk_add_qubits(self._h, n, ctypes.byref(first)))
        return first.value

    def add_cbits(self, n: int) -> int:
        first = ctypes.c_int(0)
        self._check(_lib.qk_add_cbits(self._h, n, ctypes.byref(first)))
        return first.value

    def define_gate_matrix(self, u, tol: float = 1e-9) -> int:
        u = np.ascontiguousarray(np.asarray(u, dtype=np.complex128))
        k = int(round(np.log2(u.shape[0])))
        if u.shape != (1 << k, 1 << k):
            raise ValueError("matrix must be 2^k x 2^k")
        flat = np.ascontiguousarray(u.view(np.float64).reshape(-1))
        gid = ctypes.c_int(0)
        self._check(_lib.qk_define_gate_matrix(self._h, k, flat.ctypes.data_as(_DP), tol, ctypes.byref(gid)))
        return gid.value

    def define_gate_perm_mulmod(self, w: int, c: int, N: int) -> int:
        key = ("mulmod", w, c, N)
        if key not in self._perm_cache:
            gid = ctypes.c_int(0)
            self._check(_lib.qk_define_gate_perm_mulmod(self._h, w, c, N, ctypes.byref(gid)))
            self._perm_cache[key] = gid.value
        return self._perm_cache[key]

    def define_gate_perm_table(self, f) -> int:
        f = np.ascontiguousarray(np.asarray(f, dtype=np.uint64))
        w = int(round(np.log2(len(f))))
        gid = ctypes.c_int(0)
        self._check(_lib.qk_define_gate_perm_table(self._h, w, f.ctypes.data_as(_U64P), ctypes.byref(gid)))
        return gid.value

    def apply_gate(self, gate, targets: Sequence[int], controls: Sequence[int] = (), cond: Sequence[int] = (),
                   params: Sequence[float] = ()):
        gid = GATE[gate] if isinstance(gate, str) else int(gate)
        t, nt = _ints(targets)
        c, nc = _ints(controls)
        k, nk = _ints(cond)
        p = (ctypes.c_double * max(1, len(params)))(*params)
        self._check(_lib.qk_apply_gate(self._h, gid, t, nt, c, nc, k, nk, p, len(params)))

    def apply_gates(self, ops: np.ndarray):
        """A whole gate list (GATE_OP_DTYPE entries) in one call."""
        arr = np.ascontiguousarray(ops, dtype=GATE_OP_DTYPE)
        self._check(_lib.qk_apply_gates(self._h, arr.ctypes.data, len(arr)))

    def apply_modexp(self, targets: Sequence[int], controls: Sequence[int], multipliers: Sequence[int], N: int,
                     cond: Sequence[int] = ()):
        """Multiply the register (targets, first = MSB) by the product of the
        multipliers whose control qubits are 1, mod N, in one pass."""
        if len(controls) != len(multipliers):
            raise ValueError("one multiplier per control")
        t, nt = _ints(targets)
        c, nc = _ints(controls)
        k, nk = _ints(cond)
        m = (ctypes.c_uint64 * max(1, len(multipliers)))(*[int(x) for x in multipliers])
        self._check(_lib.qk_apply_modexp(self._h, t, nt, c, m, nc, int(N), k, nk))

    def apply_rphase_cbits(self, target: int, cbits: Sequence[int]):
        cb, n = _ints(cbits)
        self._check(_lib.qk_apply_rphase_cbits(self._h, target, cb, n))

    def apply_kitaev_stage(self, control: int, perm_gate: int, targets: Sequence[int], phase_cbits: Sequence[int],
                           uniform: float, dest_cbit: int):
        t, nt = _ints(targets)
        cb, ncb = _ints(phase_cbits)
        self._check(_lib.qk_apply_kitaev_stage(self._h, control, perm_gate, t, nt, cb, ncb, uniform, dest_cbit))

    def measure(self, qubits: Sequence[int], uniforms: Sequence[float], dest: Optional[Sequence[int]] = None,
                wait: bool = True) -> Optional[int]:
        q, nq = _ints(qubits)
        u = (ctypes.c_double * max(1, nq))(*uniforms)
        d = _ints(dest)[0] if dest else None
        out = ctypes.c_uint64(0)
        self._check(_lib.qk_measure(self._h, q, nq, u, d, ctypes.byref(out) if wait else None))
        return out.value if wait else None

    def read_cbits(self, n: Optional[int] = None) -> np.ndarray:
        n = self.n_cbits if n is None else n
        buf = np.zeros(max(1, n), dtype=np.uint8)
        self._check(_lib.qk_read_cbits(self._h, buf.ctypes.data_as(_U8P), n))
        return buf[:n]

    def write_cbits(self, first: int, values: Sequence[int]):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.uint8))
        self._check(_lib.qk_write_cbits(self._h, first, v.ctypes.data_as(_U8P), len(v)))

    def get_state(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        n = self.n_qubits
        if out is None:
            out = np.empty(1 << n, dtype=self.cdtype)
        self._check(_lib.qk_get_state(self._h, out.ctypes.data, out.nbytes))
        return out

    def set_state(self, psi: np.ndarray):
        psi = np.ascontiguousarray(np.asarray(psi, dtype=self.cdtype))
        self._check(_lib.qk_set_state(self._h, psi.ctypes.data, psi.nbytes))

    def reset(self):
        self._check(_lib.qk_reset(self._h))

    def device_state(self) -> Tuple[int, int]:
        p = _P()
        nb = ctypes.c_size_t(0)
        self._check(_lib.qk_device_state(self._h, ctypes.byref(p), ctypes.byref(nb)))
        return p.value, nb.value

    def torch_view(self):
        """The device state as a torch tensor (no copy, logical qubit order)."""
        import torch

        ptr, nb = self.device_state()
        elem = 8 if self.precision == "c64" else 16

        class _Arr:
            __cuda_array_interface__ = {
                "shape": (nb // elem,), "typestr": "<c8" if elem == 8 else "<c16",
                "data": (ptr, False), "version": 3, "strides": None,
            }
        return torch.as_tensor(_Arr(), device="cuda")

    def flush(self):
        self._check(_lib.qk_flush(self._h))

    def sync(self):
        self._check(_lib.qk_sync(self._h))

    def selftest_timeout(self):
        """Enqueue the bounded-wait self-test; the next sync raises QK_ETIMEOUT."""
        self._check(_lib.qk_selftest_timeout(self._h))

    def capture_begin(self):
        self._check(_lib.qk_capture_begin(self._h))

    def capture_end(self) -> "Graph":
        g = _P()
        self._check(_lib.qk_capture_end(self._h, ctypes.byref(g)))
        return Graph(self, g)

    def counters(self) -> Dict[str, int]:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(_lib.qk_get_counters(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"launches": a.value, "state_passes": b.value, "algorithmic_bytes": c.value}

    def reset_counters(self):
        self._check(_lib.qk_reset_counters(self._h))

    def profile(self) -> Dict[str, Dict[str, float]]:
        L = (ctypes.c_uint64 * NUM_LAUNCH_CLASSES)()
        M = (ctypes.c_double * NUM_LAUNCH_CLASSES)()
        B = (ctypes.c_double * NUM_LAUNCH_CLASSES)()
        self._check(_lib.qk_profile(self._h, L, M, B))
        return {LAUNCH_CLASSES[k]: {"launches": int(L[k]), "ms": M[k], "bytes": B[k]}
                for k in range(NUM_LAUNCH_CLASSES)}


class Graph:
    """A captured CUDA graph of libqk calls on one context (qk_capture_end)."""

    def __init__(self, ctx: Context, handle):
        self._ctx = ctx
        self._g = handle

    def launch(self):
        self._ctx._check(_lib.qk_graph_launch(self._g))

    def close(self):
        if getattr(self, "_g", None):
            _lib.qk_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many circuits in few launches (qk_batch_*): circuits of at most
    SMEM_QUBITS qubits run whole in shared memory (any op), larger ones up to
    MAX_QUBITS (unitary gates, at most one control) as batched tile passes."""

    SMEM_QUBITS = 13
    MAX_QUBITS = 24

    def __init__(self, stream: Optional[int] = None):
        h = _P()
        st = _lib.qk_batch_create(ctypes.byref(h), _P(stream) if stream else None)
        if st != QK_OK:
            raise QKError(st, "qk_batch_create failed")
        self._h = h
        self._ncb: list = []
        self._n: list = []

    def _check(self, st: int):
        if st != QK_OK:
            raise QKError(st, _lib.qk_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.qk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self):
        self._check(_lib.qk_batch_clear(self._h))
        self._ncb, self._n = [], []

    def add_circuit(self, n: int, ncbits: int = 0) -> int:
        idx = ctypes.c_int(0)
        self._check(_lib.qk_batch_add_circuit(self._h, n, ncbits, ctypes.byref(idx)))
        self._ncb.append(ncbits)
        self._n.append(n)
        return idx.value

    def apply_gate(self, gate, targets, controls=(), cond=(), params=()):
        gid = GATE[gate] if isinstance(gate, str) else int(gate)
        t, nt = _ints(targets)
        c, nc = _ints(controls)
        k, nk = _ints(cond)
        p = (ctypes.c_double * max(1, len(params)))(*params)
        self._check(_lib.qk_batch_apply_gate(self._h, gid, t, nt, c, nc, k, nk, p, len(params)))

    def apply_mulmod(self, targets, controls, c: int, N: int):
        t, nt = _ints(targets)
        cl, nc = _ints(controls)
        self._check(_lib.qk_batch_apply_mulmod(self._h, t, nt, cl, nc, c, N))

    def apply_gates(self, ops: np.ndarray):
        """A whole gate list (GATE_OP_DTYPE entries) in one call."""
        arr = np.ascontiguousarray(ops, dtype=GATE_OP_DTYPE)
        self._check(_lib.qk_batch_apply_gates(self._h, arr.ctypes.data, len(arr)))

    def measure(self, qubits, uniforms, dest=None):
        q, nq = _ints(qubits)
        u = (ctypes.c_double * max(1, nq))(*uniforms)
        d = _ints(dest)[0] if dest else None
        self._check(_lib.qk_batch_measure(self._h, q, nq, u, d))

    def add_ops(self, n: int, ncbits: int, ops) -> int:
        """A workloads circuit's ops as one batch circuit (marshalling only)."""
        idx = self.add_circuit(n, ncbits)
        for op in ops:
            if op.kind == "measure":
                self.measure(op.targets, op.uniforms, op.cbits or None)
            elif op.kind == "mulmod":
                a, j, N = (int(x) for x in op.params)
                if op.cond:
                    raise ValueError("batched mul-mod takes no classical condition")
                self.apply_mulmod(op.targets, op.controls, pow(a, 1 << j, N), N)
            else:
                self.apply_gate(op.kind, op.targets, op.controls, op.cond, op.params)
        return idx

    def run(self, store_states: bool = True):
        self._check(_lib.qk_batch_run(self._h, 1 if store_states else 0))

    def done(self) -> bool:
        r = _lib.qk_batch_done(self._h)
        if r < 0:
            raise QKError(QK_ECUDA, "batch run failed")
        return r == 1

    def read(self, circuit: int, state: bool = True):
        ncb = self._ncb[circuit]
        cb = np.zeros(max(1, ncb), dtype=np.uint8)
        st = np.empty(1 << self._n[circuit], dtype=np.complex64) if state else None
        self._check(_lib.qk_batch_read(self._h, circuit, cb.ctypes.data_as(_U8P), ncb,
                                       st.ctypes.data if state else None, st.nbytes if state else 0))
        return cb[:ncb], st

    def stats(self) -> Dict[str, float]:
        """Of the last run: host planning time (ms), batched tile launches, and
        the device time (ms) after the host planning (waits for the run)."""
        ms, nl, dev = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
        self._check(_lib.qk_batch_stats(self._h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(dev)))
        return {"plan_ms": ms.value, "tile_launches": nl.value, "device_ms": dev.value}

    def read_all_cbits(self) -> np.ndarray:
        tot = sum(self._ncb)
        out = np.zeros(max(1, tot), dtype=np.uint8)
        self._check(_lib.qk_batch_read_all_cbits(self._h, out.ctypes.data_as(_U8P), tot))
        return out[:tot]


def run_ops(ctx: Context, ops) -> None:
    """Marshal a sequence of workloads.Op into libqk calls (no arithmetic on
    amplitudes here; measurements are enqueued without waiting)."""
    ops = list(ops)
    i = 0
    while i < len(ops):
        op = ops[i]
        k = op.kind
        i += 1
        if k == "mulmod" and len(op.controls) == 1 and not op.cond:
            # a run of singly controlled multiplications on one register (they
            # commute) goes to the library as one modular exponentiation
            N = int(op.params[2])
            run = [op]
            while i < len(ops):
                nx = ops[i]
                if not (nx.kind == "mulmod" and len(nx.controls) == 1 and not nx.cond and nx.targets == op.targets
                        and int(nx.params[2]) == N and nx.controls[0] not in [r.controls[0] for r in run]):
                    break
                run.append(nx)
                i += 1
            if len(run) > 1:
                ctx.apply_modexp(op.targets, [r.controls[0] for r in run],
                                 [pow(int(r.params[0]), 1 << int(r.params[1]), N) for r in run], N)
                continue
        if k == "measure":
            ctx.measure(op.targets, op.uniforms, op.cbits or None, wait=False)
        elif k == "mulmod":
            a, j, N = (int(x) for x in op.params)
            gid = ctx.define_gate_perm_mulmod(len(op.targets), pow(a, 1 << j, N), N)
            ctx.apply_gate(gid, op.targets, op.controls, op.cond)
        elif k == "rphase":
            if op.cond:
                raise ValueError("rphase takes no classical condition")
            ctx.apply_rphase_cbits(op.targets[0], op.cbits)
        elif k == "unitary":
            key = bytes(np.asarray(op.params, dtype=np.float64).tobytes())
            if key not in ctx._mat_cache:
                v = np.asarray(op.params, dtype=np.float64)
                d = int(round(np.sqrt(len(v) // 2)))
                ctx._mat_cache[key] = ctx.define_gate_matrix((v[0::2] + 1j * v[1::2]).reshape(d, d))
            ctx.apply_gate(ctx._mat_cache[key], op.targets, op.controls, op.cond)
        else:
            ctx.apply_gate(k, op.targets, op.controls, op.cond, op.params)


def run_circuit(circ, precision: str = "c64", exec_mode: str = "fused", **kw) -> Context:
    """Create a context for a workloads.Circuit and enqueue all of its ops."""
    ctx = Context(precision, exec_mode, **kw)
    ctx.add_qubits(circ.n_qubits)
    if circ.n_cbits:
        ctx.add_cbits(circ.n_cbits)
    run_ops(ctx, circ.ops)
    return ctx


def run_kitaev_fused(ctx: Context, circ) -> None:
    """Marshal a workloads.kitaev_circuit into one qk_apply_kitaev_stage call per
    stage (the op list must have the H / mulmod / rphase / H / measure / X shape
    that workloads.kitaev_circuit writes)."""
    ops = circ.ops
    i = 0
    if ops[0].kind == "x" and not ops[0].cond:  # work register initialisation
        ctx.apply_gate("x", ops[0].targets)
        i = 1
    while i < len(ops):
        h, mm = ops[i], ops[i + 1]
        has_phase = ops[i + 2].kind == "rphase"
        ph = ops[i + 2] if has_phase else None
        k = i + 3 if has_phase else i + 2
        meas = ops[k + 1]
        if h.kind != "h" or mm.kind != "mulmod" or ops[k].kind != "h" or meas.kind != "measure" or \
                ops[k + 2].kind != "x":
            raise ValueError("op list is not a sequence of Kitaev stages")
        a, j, N = (int(x) for x in mm.params)
        gid = ctx.define_gate_perm_mulmod(len(mm.targets), pow(a, 1 << j, N), N)
        ctx.apply_kitaev_stage(h.targets[0], gid, mm.targets, ph.cbits if ph else (), meas.uniforms[0],
                               meas.cbits[0])
        i = k + 3

