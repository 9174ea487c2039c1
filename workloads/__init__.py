"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and bench.py.

This module only *describes* circuits: it draws random numbers and lays out gate
lists.  It holds none of the simulation arithmetic (no gate matrices, no state
updates, no modular multiplication); each consumer turns an ``Op`` into work with
its own code.

Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), uniform doubles as ``(x >> 11) * 2**-53``.  The paper
only says that measurement follows random statistical probabilities (Circuit
section), so the generator and the way a uniform decides an outcome are this
project's reading: outcome 0 iff ``u < P0``.

Circuit recipes follow the paper's command scripts (Appendix A) and the
workload shapes of the benchmark configurations:

* ``plain_c128_circuit``  -- 12 qubits, H on all, 200 gates of alternating random
  U3 / CNOT-chain layers, the paper's QFT sequence, measure every qubit.
* ``layered_circuit``     -- n qubits (30 / 33 at full size), 500 gates of
  alternating U3-on-all / CZ-even / CZ-odd layers, then the QFT sequence.
* ``kitaev_circuit``      -- Kitaev's one-recycled-control-qubit order finding
  (the ``nx2n`` branch of Appendix A): 2b stages of H, controlled
  x -> a^(2^j) x mod N, semiclassical phase correction, H, measure, copy, reset.
* ``shor_3nx1_circuit``   -- conventional order finding (the ``3nx1`` branch):
  H on a 2b-qubit control register, controlled modular multiplications on a
  b-qubit work register, measure the work register, QFT, measure the controls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator (Steele, Lea & Flood 2014)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, n: int) -> int:
        """Integer in [0, n) (rejection sampling, no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < lim:
                return x % n

    def angle(self) -> float:
        """Angle drawn from U[0, 2 pi)."""
        return 2.0 * math.pi * self.uniform()


@dataclass(frozen=True)
class Op:
    """One circuit operation.

    kind       -- 'h', 'x', 'y', 'z', 's', 'sdg', 't', 'u3', 'p', 'swap', 'unitary',
                  'mulmod', 'rphase', 'measure'
    targets    -- target qubits; for registers the first-listed qubit is the most
                  significant bit of the register value
    controls   -- quantum controls (all must be |1>)
    params     -- gate angles; for 'mulmod' (a, j, N) meaning x -> a^(2^j) x mod N;
                  for 'unitary' the flat row-major interleaved (re, im) matrix
    cond       -- classical condition: cbits that must all be 1 for the op to act
    cbits      -- 'rphase': cbits read, most recent first;  'measure': destination
                  cbits (one per measured qubit) or empty
    uniforms   -- 'measure': one uniform per measured qubit, in list order
    """

    kind: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    params: Tuple[float, ...] = ()
    cond: Tuple[int, ...] = ()
    cbits: Tuple[int, ...] = ()
    uniforms: Tuple[float, ...] = ()


@dataclass
class Circuit:
    n_qubits: int
    n_cbits: int
    ops: List[Op] = field(default_factory=list)
    name: str = ""

    def gate_count(self) -> int:
        """Number of gate ops (measurements and SWAPs included, as the paper counts commands)."""
        return sum(1 for op in self.ops if op.kind != "measure")


# ---------------------------------------------------------------------------
# gate-list builders
# ---------------------------------------------------------------------------

def qft_ops(qubits: Sequence[int]) -> List[Op]:
    """QFT command sequence of Appendix A (the 3nx1 branch): for each qubit c in
    order, H(c) then CPHASE(d, c) with phi = pi / 2^(i+1) for the i-th later qubit d;
    finally SWAP the register end for end.  qubits[0] is the register MSB."""
    ops: List[Op] = []
    q = list(qubits)
    nq = len(q)
    for c in range(nq):
        ops.append(Op("h", (q[c],)))
        for i, d in enumerate(range(c + 1, nq)):
            ops.append(Op("p", (q[c],), controls=(q[d],), params=(math.pi / float(1 << (i + 1)),)))
    for i in range(nq // 2):
        ops.append(Op("swap", (q[i], q[nq - 1 - i])))
    return ops


def _u3_op(rng: SplitMix64, q: int) -> Op:
    return Op("u3", (q,), params=(rng.angle(), rng.angle(), rng.angle()))


def plain_c128_circuit(seed: int = 1, n: int = 12, n_gates: int = 200, measure: bool = True) -> Circuit:
    """12-qubit complex128 workload: H on every qubit, then exactly ``n_gates`` gates
    of alternating [U3 on q0..n-1] / [CNOT 0->1, 1->2, ...] layers (the last layer
    truncated), the QFT sequence, then measure q0..n-1 in order with seeded uniforms."""
    rng = SplitMix64(seed)
    ops = [Op("h", (q,)) for q in range(n)]
    count = 0
    layer = 0
    while count < n_gates:
        if layer % 2 == 0:
            for q in range(n):
                if count == n_gates:
                    break
                ops.append(_u3_op(rng, q))
                count += 1
        else:
            for q in range(n - 1):
                if count == n_gates:
                    break
                ops.append(Op("x", (q + 1,), controls=(q,)))
                count += 1
        layer += 1
    ops += qft_ops(range(n))
    n_cb = 0
    if measure:
        ops.append(Op("measure", tuple(range(n)), cbits=tuple(range(n)),
                      uniforms=tuple(rng.uniform() for _ in range(n))))
        n_cb = n
    return Circuit(n, n_cb, ops, name=f"plain{n}q_c128_seed{seed}")


def layered_circuit(n: int, seed: int = 2, n_gates: int = 500, qft: bool = True,
                    measure: int = 0) -> Circuit:
    """Single-large-state workload: |0...0>, then exactly ``n_gates`` gates of
    repeating [U3 on every qubit] [CZ (0,1),(2,3),...] [CZ (1,2),(3,4),...] layers
    (the last layer truncated), then the QFT sequence on all n qubits.  With
    ``measure`` > 0 the first ``measure`` qubits are measured at the end."""
    rng = SplitMix64(seed)
    ops: List[Op] = []
    count = 0
    layer = 0
    while count < n_gates:
        kind = layer % 3
        if kind == 0:
            for q in range(n):
                if count == n_gates:
                    break
                ops.append(_u3_op(rng, q))
                count += 1
        else:
            start = 0 if kind == 1 else 1
            for q in range(start, n - 1, 2):
                if count == n_gates:
                    break
                ops.append(Op("z", (q + 1,), controls=(q,)))
                count += 1
        layer += 1
    if qft:
        ops += qft_ops(range(n))
    n_cb = 0
    if measure:
        ops.append(Op("measure", tuple(range(measure)), cbits=tuple(range(measure)),
                      uniforms=tuple(rng.uniform() for _ in range(measure))))
        n_cb = measure
    return Circuit(n, n_cb, ops, name=f"layered{n}q_{n_gates}g_seed{seed}")


def batch_layer_spec(index: int, seed: int = 4, n_min: int = 10, n_max: int = 20,
                     d_min: int = 50, d_max: int = 300):
    """One circuit of the batched workload: n ~ U{n_min..n_max} qubits, depth ~
    U{d_min..d_max} layers, each layer U3(theta, phi, lambda ~ U[0, 2 pi)) on every
    qubit then CZ on the even (even layers) or odd (odd layers) neighbour pairs.
    Returns (n, depth, angles[depth, n, 3]); numpy's PCG64 keyed by (seed, index)
    keeps thousands of circuits cheap to draw."""
    import numpy as np

    rng = np.random.Generator(np.random.PCG64([seed, index]))
    n = int(rng.integers(n_min, n_max + 1))
    depth = int(rng.integers(d_min, d_max + 1))
    angles = rng.uniform(0.0, 2.0 * math.pi, size=(depth, n, 3))
    return n, depth, angles


def layer_spec_circuit(n: int, depth: int, angles) -> Circuit:
    """The ops of a batch_layer_spec circuit (for the oracle and per-gate paths)."""
    ops: List[Op] = []
    for L in range(depth):
        ops += [Op("u3", (q,), params=tuple(float(a) for a in angles[L][q])) for q in range(n)]
        ops += [Op("z", (q + 1,), controls=(q,)) for q in range(L % 2, n - 1, 2)]
    return Circuit(n, 0, ops, name=f"layers{n}q_{depth}d")


# ---------------------------------------------------------------------------
# Kitaev order finding inputs
# ---------------------------------------------------------------------------

def _is_probable_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (bases of Sorenson & Webster 2015)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _is_prime_power(n: int) -> bool:
    for k in range(2, n.bit_length() + 1):
        r = round(n ** (1.0 / k))
        for c in (r - 1, r, r + 1):
            if c > 1 and c ** k == n:
                return True
    return False


def kitaev_parameters(b: int, seed: int = 3) -> Tuple[int, int]:
    """Seeded random odd b-bit composite N (not a prime power) and a base a with
    gcd(a, N) = 1 and a != 1 (so the order of a mod N exceeds 1)."""
    if b < 4:
        raise ValueError("need b >= 4 for an odd composite")
    rng = SplitMix64(seed * 1000003 + b)
    while True:
        N = (1 << (b - 1)) | rng.below(1 << (b - 1)) | 1
        if _is_probable_prime(N) or _is_prime_power(N):
            continue
        while True:
            a = 2 + rng.below(N - 3)
            if math.gcd(a, N) == 1:
                return N, a


def kitaev_circuit(N: int, a: int, t: int | None = None, seed: int = 3,
                   uniforms: Sequence[float] | None = None) -> Circuit:
    """Kitaev's one-control-qubit order finding (the nx2n branch of Appendix A).

    Qubit 0 is the recycled control; qubits 1..b hold the work register (qubit 1 the
    MSB), b = bit_length(N).  Stage e (e = 0..t-1) uses j = t-1-e:
    H(0); controlled x -> a^(2^j) x mod N on 1..b; phase correction on qubit 0 from
    cbits e-1..0 (most recent first); H(0); measure 0 into cbit e; X(0) if cbit e.
    ``t`` defaults to 2b (one reading of the stage count; the paper's script uses
    bit_length(N^2 - 1), which is 2b or 2b-1)."""
    b = N.bit_length()
    if t is None:
        t = 2 * b
    rng = SplitMix64(seed * 7919 + N)
    if uniforms is None:
        uniforms = [rng.uniform() for _ in range(t)]
    if len(uniforms) != t:
        raise ValueError("need one uniform per stage")
    reg = tuple(range(1, b + 1))
    ops: List[Op] = [Op("x", (b,))]
    for e in range(t):
        j = t - 1 - e
        ops.append(Op("h", (0,)))
        ops.append(Op("mulmod", reg, controls=(0,), params=(a, j, N)))
        if e > 0:
            ops.append(Op("rphase", (0,), cbits=tuple(range(e - 1, -1, -1))))
        ops.append(Op("h", (0,)))
        ops.append(Op("measure", (0,), cbits=(e,), uniforms=(uniforms[e],)))
        ops.append(Op("x", (0,), cond=(e,)))
    return Circuit(b + 1, t, ops, name=f"kitaev_N{N}_a{a}_t{t}")


def paper_stage_count(N: int) -> int:
    """nC of the paper's script: bit_length(N^2 - 1) (Appendix A, nx2n branch)."""
    return (N * N - 1).bit_length()


def shor_3nx1_circuit(N: int, a: int, t: int | None = None, seed: int = 5,
                      uniforms: Sequence[float] | None = None) -> Circuit:
    """Conventional Shor order finding, the 3nx1 branch of Appendix A.

    Qubits 0..t-1 form the control register (qubit 0 its MSB), qubits t..t+b-1 the
    work register (qubit t its MSB), b = bit_length(N) and t = bit_length(N^2 - 1)
    by default.  Steps: X on the last qubit (work register = 1); H on every
    control qubit; for c = 0..t-1 the controlled x -> a^(2^c) x mod N on the work
    register, controlled by qubit t-1-c (so the exponent reads with qubit 0 as its
    MSB); measure the work register (qubit by qubit, into cbits 0..b-1); the QFT
    command sequence of Appendix A on the control register (H then CPHASE pi/2^(i+1),
    then the end-for-end SWAPs); finally measure the control register into cbits
    b..b+t-1 (qubit 0 into cbit b), which the script leaves to the viewer."""
    b = N.bit_length()
    if t is None:
        t = paper_stage_count(N)
    n = t + b
    rng = SplitMix64(seed * 104729 + N)
    if uniforms is None:
        uniforms = [rng.uniform() for _ in range(b + t)]
    if len(uniforms) != b + t:
        raise ValueError("need one uniform per measured qubit")
    ctrl = tuple(range(t))
    work = tuple(range(t, n))
    ops: List[Op] = [Op("x", (n - 1,))]
    ops += [Op("h", (q,)) for q in ctrl]
    for c in range(t):
        ops.append(Op("mulmod", work, controls=(t - 1 - c,), params=(a, c, N)))
    ops.append(Op("measure", work, cbits=tuple(range(b)), uniforms=tuple(uniforms[:b])))
    ops += qft_ops(ctrl)
    ops.append(Op("measure", ctrl, cbits=tuple(range(b, b + t)), uniforms=tuple(uniforms[b:])))
    return Circuit(n, b + t, ops, name=f"shor3nx1_N{N}_a{a}_t{t}")


def serving_request(seed: int, n: int | None = None, n_min: int = 8, n_max: int = 33) -> Circuit:
    """One serving request: n qubits (log-uniform in [n_min, n_max] unless given),
    5..40 layers cycling U3-on-every-qubit / CZ-even / CZ-odd, one controlled
    x -> a^(2^j) x mod N oracle on a w-qubit register (w in 10..16, only when
    n >= w + 1: control qubit 0, register qubits 1..w with qubit 1 the MSB), and
    1..4 mid-circuit measurements, each into its own cbit and followed by a U3 on
    another qubit conditioned on that cbit."""
    rng = SplitMix64(seed * 2654435761 + 17)
    if n is None:
        n = int(round(math.exp(math.log(n_min) + rng.uniform() * (math.log(n_max) - math.log(n_min)))))
    n_layers = 5 + rng.below(36)
    w = 10 + rng.below(7)
    oracle_at = rng.below(n_layers) if n >= w + 1 else -1
    n_meas = 1 + rng.below(4)
    meas_at = sorted(rng.below(n_layers) for _ in range(n_meas))
    ops: List[Op] = []
    k = 0
    for layer in range(n_layers):
        kind = layer % 3
        if kind == 0:
            ops += [_u3_op(rng, q) for q in range(n)]
        else:
            start = 0 if kind == 1 else 1
            ops += [Op("z", (q + 1,), controls=(q,)) for q in range(start, n - 1, 2)]
        if layer == oracle_at:
            while True:
                N = (1 << (w - 1)) | rng.below(1 << (w - 1)) | 1
                a = 2 + rng.below(N - 3)
                if math.gcd(a, N) == 1:
                    break
            ops.append(Op("mulmod", tuple(range(1, w + 1)), controls=(0,), params=(a, rng.below(2 * w), N)))
        while k < n_meas and meas_at[k] == layer:
            q = rng.below(n)
            t = (q + 1 + rng.below(n - 1)) % n
            ops.append(Op("measure", (q,), cbits=(k,), uniforms=(rng.uniform(),)))
            ops.append(Op("u3", (t,), params=(rng.angle(), rng.angle(), rng.angle()), cond=(k,)))
            k += 1
    return Circuit(n, n_meas, ops, name=f"request{seed}_n{n}")


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 7):
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = SplitMix64(seed)
    t, out = 0.0, []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        out.append(t)
    return out


def random_state(n: int, seed: int):
    """Seeded random normalised complex128 state (numpy array) for parity inputs:
    independent standard normal real and imaginary parts (numpy PCG64), normalised."""
    import numpy as np

    g = np.random.Generator(np.random.PCG64(seed))
    v = g.standard_normal(2 * (1 << n))
    psi = v[0::2] + 1j * v[1::2]
    psi /= np.linalg.norm(psi)
    return psi.astype(np.complex128)
