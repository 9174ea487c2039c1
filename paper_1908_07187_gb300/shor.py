"""Classical post-processing of an order-finding run (host arithmetic only).

The Shor section of the paper turns the classical bits of an order-finding run
(Kitaev's, or the conventional 3nx1 circuit's control register) into the order
r of a modulo N by continued fractions, then into prime factors.  Here: the t
measured bits give y (Kitaev: y = sum_e m_e 2^e, stage e's bit is m_e; 3nx1: the
control register's value, qubit 0 its MSB), y / 2^t is
close to s / r for some s, so r (or a divisor of it when gcd(s, r) > 1) is a
denominator of a convergent of y / 2^t; a small multiple of that denominator is
tried until a^r = 1 mod N (the paper's third 24-bit run found 141210 = r / 4).
If r is even and a^(r/2) != -1 mod N, gcd(a^(r/2) +- 1, N) are nontrivial
factors.
"""
from __future__ import annotations

from math import gcd
from typing import List, Optional, Sequence, Tuple


def outcome_from_bits(bits: Sequence[int]) -> int:
    """y = sum_e m_e 2^e from the stage bits m_0, m_1, ... (Kitaev's run: stage e
    measures bit e of y)."""
    return sum((int(m) & 1) << e for e, m in enumerate(bits))


def register_from_bits(bits: Sequence[int]) -> int:
    """Value of a register measured qubit by qubit in list order, the first-listed
    qubit its MSB (the 3nx1 run's control and work registers)."""
    v = 0
    for m in bits:
        v = (v << 1) | (int(m) & 1)
    return v


def convergents(num: int, den: int) -> List[Tuple[int, int]]:
    """Convergents p/q of the continued fraction of num/den (den > 0), in order."""
    if den <= 0:
        raise ValueError("denominator must be positive")
    out: List[Tuple[int, int]] = []
    p0, q0, p1, q1 = 0, 1, 1, 0          # h_{-2}/k_{-2}, h_{-1}/k_{-1}
    a, b = num, den
    while b:
        c = a // b
        p0, p1 = p1, c * p1 + p0
        q0, q1 = q1, c * q1 + q0
        out.append((p1, q1))
        a, b = b, a - c * b
    return out


def order_candidates(y: int, t: int, N: int) -> List[int]:
    """Distinct denominators q < N of the convergents of y / 2^t, smallest first."""
    seen, out = set(), []
    for _, q in convergents(y, 1 << t):
        if 1 < q < N and q not in seen:
            seen.add(q)
            out.append(q)
    return out


def order_from_outcome(y: int, t: int, a: int, N: int, max_multiple: int = 16) -> Optional[int]:
    """The order r of a mod N read from one outcome y of a t-stage run, or None.

    Each convergent denominator q, then its multiples k q (k <= max_multiple), is
    tested for a^(k q) = 1 mod N; the first hit is returned."""
    if gcd(a, N) != 1:
        raise ValueError("a and N must be coprime")
    for q in order_candidates(y, t, N):
        for k in range(1, max_multiple + 1):
            r = k * q
            if r >= N:
                break
            if pow(a, r, N) == 1:
                return r
    return None


def factors_from_order(a: int, r: int, N: int) -> Optional[Tuple[int, int]]:
    """Nontrivial factors (f, N // f) from an even order r, or None."""
    if r % 2 or pow(a, r, N) != 1:
        return None
    h = pow(a, r // 2, N)
    if h == N - 1:
        return None
    for f in (gcd(h - 1, N), gcd(h + 1, N)):
        if 1 < f < N:
            return (min(f, N // f), max(f, N // f))
    return None
