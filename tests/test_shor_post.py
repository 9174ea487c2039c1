"""Host post-processing of order finding (continued fractions, factors): pinned
by textbook continued fractions, brute-force orders and the paper's printed
24-bit values."""
import os
import sys
from math import gcd

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from conftest import load_golden  # noqa: E402
from paper_1908_07187_gb300 import shor  # noqa: E402


def brute_order(a, N):
    x, k = a % N, 1
    while x != 1:
        x = x * a % N
        k += 1
    return k


def test_convergents_textbook():
    # 415/93 = [4; 2, 6, 7]: convergents 4, 9/2, 58/13, 415/93
    assert shor.convergents(415, 93) == [(4, 1), (9, 2), (58, 13), (415, 93)]
    # every convergent of a rational ends at the fraction in lowest terms
    assert shor.convergents(64, 256)[-1] == (1, 4)


def test_outcome_bit_order():
    assert shor.outcome_from_bits([0, 1, 1]) == 6
    assert shor.outcome_from_bits([]) == 0


@pytest.mark.parametrize("y,expect", [(64, 4), (192, 4), (128, 4), (0, None)])
def test_n15_a7(y, expect):
    # t = 8 stages: the phases are s/4, so y is a multiple of 64 (s = 0 fails)
    r = shor.order_from_outcome(y, 8, 7, 15)
    assert r == expect
    if r:
        assert shor.factors_from_order(7, r, 15) == (3, 5)


def test_paper_24bit_order_from_a_quarter_phase():
    g = load_golden("paper_values.txt")
    N, r_true, part = g["n13564597"], g["n13564597_order"], g["n13564597_partial"]
    assert r_true == 4 * part
    t = 2 * N.bit_length()
    # a phase s / r with gcd(s, r) = 4 gives the convergent denominator r / 4
    y = round(4 * 2 ** t / r_true)
    assert part in shor.order_candidates(y, t, N)
    assert shor.order_from_outcome(y, t, 2, N) == r_true
    assert pow(2, r_true, N) == 1


@pytest.mark.parametrize("N,a", [(21, 2), (35, 3), (187, 5), (3127, 7)])
def test_every_peak_gives_a_multiple_of_the_order(N, a):
    r = brute_order(a, N)
    t = 2 * N.bit_length()
    for s in range(r):
        y = round(s * 2 ** t / r) % (1 << t)
        got = shor.order_from_outcome(y, t, a, N)
        if gcd(s, r) == 1:
            assert got == r          # coprime s: the order itself
        if got is not None:
            assert got % r == 0 and pow(a, got, N) == 1


def test_factors_need_an_even_order_without_minus_one():
    assert shor.factors_from_order(2, 4, 15) == (3, 5)
    assert shor.factors_from_order(14, 2, 15) is None      # 14 = -1 mod 15
    assert shor.factors_from_order(4, 3, 21) is None       # odd order
    with pytest.raises(ValueError):
        shor.order_from_outcome(1, 4, 3, 15)
