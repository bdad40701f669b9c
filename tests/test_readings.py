"""Arithmetic behind the operation-count reading (Section 3.4.5 and Section
3.3): the per-iteration tables summed over k = 1..q with m = p b, n = q b.

The tiled table sums to a form that differs from the printed T_tiled in the
n^3 r / b coefficient (-1/6, printed -5/6) and in two lower terms; the
blocked table sums exactly to the printed T_blocked.
"""
import pytest

sp = pytest.importorskip("sympy")


def _symbols():
    return sp.symbols("b r k m n", positive=True)


def test_tiled_table_sum_and_the_printed_form():
    b, r, k, m, n = _symbols()
    p, q = m / b, n / b
    table = sp.summation((p - k + 1) * b**3 + (p - k + 1) * (q - k) * b**2 * r, (k, 1, q))
    printed = sp.Rational(1, 6) * (6 * m * n * b + 3 * n * b**2 + 3 * m * n**2 * r / b - 3 * n**2 * b
                                   - 5 * n**3 * r / b - 3 * m * n * r)
    ours = (m * n * b + n * b**2 / 2 - n**2 * b / 2 + m * n**2 * r / (2 * b) - n**3 * r / (6 * b)
            - m * n * r / 2 + n**2 * r / 2 - n * b * r / 3)
    assert sp.simplify(table - ours) == 0
    assert sp.simplify(table - printed) != 0
    # p = q = 2 by hand: k = 1 gives 2b^3 + 2b^2 r, k = 2 gives b^3
    at2 = {m: 2 * b, n: 2 * b}
    assert sp.simplify(table.subs(at2) - (3 * b**3 + 2 * b**2 * r)) == 0
    assert sp.simplify(printed.subs(at2) - (3 * b**3 - sp.Rational(14, 3) * b**2 * r)) == 0


def test_blocked_table_sum_is_the_printed_form():
    b, r, k, m, n = _symbols()
    p, q = m / b, n / b
    table = sp.summation(b**3 + p * b**2 * r + (q - k) * (b**2 * r + p * b * r**2), (k, 1, q))
    printed = sp.Rational(1, 2) * (2 * n * b**2 + 2 * m * n * r + n**2 * r + m * n**2 * r**2 / b**2
                                   - n * b * r - m * n * r**2 / b)
    assert sp.simplify(table - printed) == 0
