"""Plain complex128 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The product path
(``paper_1908_07187_gb300``) never imports it, and it imports nothing from the
product.  The arithmetic lives in ``qk_oracle.c`` (one plain loop per operation,
double precision); this file holds the textbook gate matrices, the driver that
walks a ``workloads.Circuit`` op by op, and Kitaev's order finding in the order of
the paper's command script (Appendix A, nx2n branch).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(Kronecker-product brute force, the DFT closed form, Bell/GHZ states, the
closed-form phase-estimation distribution, printed values of the paper).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile qk_oracle.c into liboracle.so next to it (gcc, portable flags).
    With openmp=True, the all-core build liboracle_omp.so (-fopenmp: the gate
    loop's groups split across the host's cores; nothing else differs), used
    only to time the oracle on every core."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC"] +
                              (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            L = ctypes.CDLL(build(openmp=openmp))
            dp, ip, up = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64)
            L.orc_apply_unitary.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp, ip, ctypes.c_int]
            L.orc_apply_perm.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, up, ip, ctypes.c_int]
            L.orc_apply_mulmod.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ctypes.c_uint64,
                                           ctypes.c_uint64, ip, ctypes.c_int]
            L.orc_prob0.argtypes = [dp, ctypes.c_int, ctypes.c_int]
            L.orc_prob0.restype = ctypes.c_double
            L.orc_measure.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
            L.orc_apply_rphase.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte),
                                           ctypes.c_int]
            L.orc_norm2.argtypes = [dp, ctypes.c_int]
            L.orc_norm2.restype = ctypes.c_double
            _libs[openmp] = L
    return _libs[openmp]


def _ints(xs: Sequence[int]):
    arr = (ctypes.c_int * max(1, len(xs)))(*xs)
    return arr


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# textbook gate matrices (row/column index = register value, first target = MSB)
# ---------------------------------------------------------------------------
SQ2 = 1.0 / math.sqrt(2.0)
GATES_1Q: Dict[str, np.ndarray] = {
    "h": np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=np.complex128),
    "x": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
    "s": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "sdg": np.array([[1, 0], [0, -1j]], dtype=np.complex128),
    "t": np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128),
    "tdg": np.array([[1, 0], [0, np.exp(-1j * math.pi / 4)]], dtype=np.complex128),
}


def rz(theta: float) -> np.ndarray:
    """Rotation about Z, exp(-i theta Z / 2) = diag(e^{-i theta/2}, e^{i theta/2})."""
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]], dtype=np.complex128)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    """OpenQASM 2 U(theta, phi, lambda) (Cross et al. 2017)."""
    c, s = math.cos(theta / 2.0), math.sin(theta / 2.0)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def phase(phi: float) -> np.ndarray:
    """diag(1, e^{i phi}); with one control this is CPHASE (Appendix A)."""
    return np.array([[1, 0], [0, np.exp(1j * phi)]], dtype=np.complex128)


SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def gate_matrix(kind: str, params: Sequence[float] = ()) -> np.ndarray:
    if kind in GATES_1Q:
        return GATES_1Q[kind]
    if kind == "u3":
        return u3(*params)
    if kind == "p":
        return phase(params[0])
    if kind == "rz":
        return rz(params[0])
    if kind == "swap":
        return SWAP
    if kind == "unitary":
        v = np.asarray(params, dtype=np.float64)
        d = int(round(math.sqrt(len(v) // 2)))
        return (v[0::2] + 1j * v[1::2]).reshape(d, d)
    raise ValueError(f"no matrix for gate kind {kind!r}")


# ---------------------------------------------------------------------------
# state
# ---------------------------------------------------------------------------
class OracleState:
    """A 2^n complex128 state vector plus a classical bit register."""

    def __init__(self, n: int, n_cbits: int = 0, psi: Optional[np.ndarray] = None, openmp: bool = False):
        self.n = n
        self._openmp = openmp
        if psi is None:
            self.psi = np.zeros(1 << n, dtype=np.complex128)
            self.psi[0] = 1.0
        else:
            psi = np.ascontiguousarray(psi, dtype=np.complex128)
            if psi.shape != (1 << n,):
                raise ValueError("state length must be 2^n")
            self.psi = psi.copy()
        self.cbits = np.zeros(n_cbits, dtype=np.uint8)
        self.last_p0: List[float] = []

    # Q-Kit "AddQubits": new qubits start in |0> and become the highest index bits.
    def add_qubits(self, k: int) -> int:
        first = self.n
        new = np.zeros(1 << (self.n + k), dtype=np.complex128)
        new[: 1 << self.n] = self.psi
        self.psi, self.n = new, self.n + k
        return first

    def add_cbits(self, k: int) -> int:
        first = len(self.cbits)
        self.cbits = np.concatenate([self.cbits, np.zeros(k, dtype=np.uint8)])
        return first

    def _cond(self, cond: Sequence[int]) -> bool:
        return all(self.cbits[c] == 1 for c in cond)

    def apply_matrix(self, u: np.ndarray, targets: Sequence[int], controls: Sequence[int] = ()):
        u = np.ascontiguousarray(u, dtype=np.complex128)
        k = len(targets)
        if u.shape != (1 << k, 1 << k):
            raise ValueError("matrix shape does not match target count")
        flat = np.ascontiguousarray(u.view(np.float64).reshape(-1))
        rc = lib(self._openmp).orc_apply_unitary(_dptr(self.psi.view(np.float64)), self.n, k, _ints(targets),
                                     _dptr(flat), _ints(controls), len(controls))
        if rc != 0:
            raise ValueError("oracle rejected unitary arguments")

    def apply_perm(self, f: Sequence[int], targets: Sequence[int], controls: Sequence[int] = ()):
        arr = np.ascontiguousarray(np.asarray(f, dtype=np.uint64))
        rc = lib().orc_apply_perm(_dptr(self.psi.view(np.float64)), self.n, len(targets), _ints(targets),
                                  arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ints(controls),
                                  len(controls))
        if rc != 0:
            raise ValueError("oracle rejected permutation (not a bijection or bad qubits)")

    def apply_mulmod(self, c: int, N: int, targets: Sequence[int], controls: Sequence[int] = ()):
        rc = lib().orc_apply_mulmod(_dptr(self.psi.view(np.float64)), self.n, len(targets), _ints(targets),
                                    c, N, _ints(controls), len(controls))
        if rc != 0:
            raise ValueError("oracle rejected mul-mod arguments")

    def prob0(self, q: int) -> float:
        return lib().orc_prob0(_dptr(self.psi.view(np.float64)), self.n, q)

    def measure(self, qubits: Sequence[int], uniforms: Sequence[float],
                dest: Sequence[int] = ()) -> int:
        """Sequential single-qubit measurements in list order, one uniform each.
        Returns the outcome as a register value (first-listed qubit = MSB)."""
        if len(uniforms) != len(qubits):
            raise ValueError("one uniform per measured qubit")
        value = 0
        self.last_p0 = []
        for idx, (q, u) in enumerate(zip(qubits, uniforms)):
            p0 = ctypes.c_double(0.0)
            m = lib().orc_measure(_dptr(self.psi.view(np.float64)), self.n, q, float(u), ctypes.byref(p0))
            if m < 0:
                raise ValueError("oracle rejected measurement arguments")
            self.last_p0.append(p0.value)
            if dest:
                self.cbits[dest[idx]] = m
            value = (value << 1) | m
        return value

    def rphase(self, target: int, cbits: Sequence[int]):
        vals = (ctypes.c_ubyte * max(1, len(cbits)))(*[int(self.cbits[c]) for c in cbits])
        rc = lib().orc_apply_rphase(_dptr(self.psi.view(np.float64)), self.n, target, vals, len(cbits))
        if rc != 0:
            raise ValueError("oracle rejected rphase arguments")

    def norm2(self) -> float:
        return lib().orc_norm2(_dptr(self.psi.view(np.float64)), self.n)

    # -- walk a workloads.Op --------------------------------------------------
    def apply_op(self, op) -> Optional[int]:
        if op.kind == "measure":
            return self.measure(op.targets, op.uniforms, op.cbits)
        if not self._cond(op.cond):
            return None
        if op.kind == "mulmod":
            a, j, N = (int(x) for x in op.params)
            self.apply_mulmod(pow(a, 1 << j, N), N, op.targets, op.controls)
        elif op.kind == "rphase":
            self.rphase(op.targets[0], op.cbits)
        else:
            self.apply_matrix(gate_matrix(op.kind, op.params), op.targets, op.controls)
        return None


def run_circuit(circ, psi0: Optional[np.ndarray] = None) -> OracleState:
    """Apply every op of a workloads.Circuit to |0...0> (or psi0)."""
    st = OracleState(circ.n_qubits, circ.n_cbits, psi0)
    for op in circ.ops:
        st.apply_op(op)
    return st


def kitaev_order_finding(N: int, a: int, t: int, uniforms: Sequence[float]):
    """Kitaev's one-recycled-qubit order finding, stage by stage as in the paper's
    nx2n script (Appendix A): qubit 0 the control, qubits 1..b the work register
    (qubit 1 the MSB) initialised to |1>.  Stage e (j = t-1-e): H(0); controlled
    x -> a^(2^j) x mod N; phase correction from cbits e-1..0; H(0); measure 0 into
    cbit e; X(0) if cbit e.  Returns (y, bits, stage P(m_e) list, final state),
    y = sum_e m_e 2^e."""
    b = N.bit_length()
    st = OracleState(b + 1, t)
    reg = list(range(1, b + 1))
    st.apply_matrix(GATES_1Q["x"], [b])
    probs = []
    for e in range(t):
        j = t - 1 - e
        st.apply_matrix(GATES_1Q["h"], [0])
        st.apply_mulmod(pow(a, 1 << j, N), N, reg, [0])
        if e > 0:
            st.rphase(0, list(range(e - 1, -1, -1)))
        st.apply_matrix(GATES_1Q["h"], [0])
        m = st.measure([0], [uniforms[e]], [e])
        p0 = st.last_p0[0]
        probs.append(p0 if m == 0 else 1.0 - p0)
        if st.cbits[e]:
            st.apply_matrix(GATES_1Q["x"], [0])
    bits = [int(x) for x in st.cbits]
    y = sum(m << e for e, m in enumerate(bits))
    return y, bits, probs, st
