"""Checks of readings of the paper that the implementation relies on.

* Operation counts (Section 3.4.5 and Section 3.3): the per-iteration
  tables summed over k = 1..q with m = p b, n = q b.  The tiled table sums
  to a form that differs from the printed T_tiled in the n^3 r / b
  coefficient (-1/6, printed -5/6) and in two lower terms; the blocked
  table sums exactly to the printed T_blocked.
* The GPU's reduced-pair trapezoidal update (reading 8) and its whole-block
  T assembled from inner blocks (reading 14): the same operators as
  Sections 3.4.3-3.4.4 and Eq. 3, in exact arithmetic.
"""
import numpy as np
import pytest

from oracle import blr_qr as O


def _symbols():
    sp = pytest.importorskip("sympy")
    return sp, sp.symbols("b r k m n", positive=True)


def test_tiled_table_sum_and_the_printed_form():
    sp, (b, r, k, m, n) = _symbols()
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
    sp, (b, r, k, m, n) = _symbols()
    p, q = m / b, n / b
    table = sp.summation(b**3 + p * b**2 * r + (q - k) * (b**2 * r + p * b * r**2), (k, 1, q))
    printed = sp.Rational(1, 2) * (2 * n * b**2 + 2 * m * n * r + n**2 * r + m * n**2 * r**2 / b**2
                                   - n * b * r - m * n * r**2 / b)
    assert sp.simplify(table - printed) == 0


# ---------------------------------------------------------------- readings 8 and 14


def _tsqrt_low_rank(rng, b, r):
    """A TSQRT reflector block with a low-rank tail: Y~ = U Y, U orthonormal."""
    rkk = np.triu(rng.standard_normal((b, b))) + 3 * np.eye(b)
    u, _ = np.linalg.qr(rng.standard_normal((b, r)))
    v = rng.standard_normal((b, r))
    _, y, t = O.tsqrt(rkk, v.T)            # y: r x b (Y_ik), t: b x b
    return u, y, t


@pytest.mark.parametrize("b,r", [(16, 3), (24, 8), (8, 8)])
def test_reduced_pair_update_equals_the_trapezoidal_reflector(b, r):
    """Reading 8: with Y~ = U Y and U orthonormal, applying Q^T =
    (I - [I; Y~] T [I; Y~]^T)^T to [R; A] only changes R and U^T A:
    P = U^T A, S = R + Y^T P, W = T^T S, R' = R - W, P' = P - Y W,
    A' = A + U (P' - P).  Same operator as Section 3.4.4, in exact
    arithmetic."""
    rng = np.random.default_rng(b + r)
    u, y, t = _tsqrt_low_rank(rng, b, r)
    rkj = rng.standard_normal((b, b))
    aij = rng.standard_normal((b, b))
    yt = u @ y
    full = np.vstack([np.eye(b), yt])
    qt = (np.eye(2 * b) - full @ t @ full.T).T
    want = qt @ np.vstack([rkj, aij])
    p = u.T @ aij
    w = t.T @ (rkj + y.T @ p)
    r_new = rkj - w
    p_new = p - y @ w
    a_new = aij + u @ (p_new - p)
    got = np.vstack([r_new, a_new])
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    # the part of A orthogonal to U is untouched
    proj = np.eye(b) - u @ u.T
    assert np.allclose(proj @ a_new, proj @ aij, atol=1e-13 * np.abs(aij).max())


@pytest.mark.parametrize("b,nb", [(16, 4), (32, 8), (24, 8)])
def test_whole_block_t_from_inner_blocks_and_gram(b, nb):
    """Reading 14: the b x b T of all b reflectors (Eq. 3) from the stored
    inner T blocks (nb reflectors each) and G = Y^T Y of the tails, block
    column by block column: T(0:J, J) = -T(0:J, 0:J) G(0:J, J) T_J.  The
    identity parts of [I; Y] are orthogonal, so G alone carries the
    off-diagonal products."""
    rng = np.random.default_rng(b * nb)
    rkk = np.triu(rng.standard_normal((b, b))) + 3 * np.eye(b)
    tail = rng.standard_normal((b, b))                     # dense tail
    _, y, t_full = O.tsqrt(rkk, tail)
    tau = np.diag(t_full)
    g = y.T @ y
    t = np.zeros((b, b))
    for j0 in range(0, b, nb):
        j1 = j0 + nb
        tj = O.t_from_gram(g[j0:j1, j0:j1], tau[j0:j1])     # the stored inner block
        t[j0:j1, j0:j1] = tj
        if j0:
            t[:j0, j0:j1] = -t[:j0, :j0] @ g[:j0, j0:j1] @ tj
    assert np.allclose(t, t_full, atol=1e-12 * np.abs(t_full).max())
    # and it is the compact WY of the explicit product of the reflectors
    full = np.vstack([np.eye(b), y])
    q = np.eye(2 * b)
    for j in range(b):
        v = full[:, j]
        q = q @ (np.eye(2 * b) - tau[j] * np.outer(v, v))
    assert np.allclose(np.eye(2 * b) - full @ t @ full.T, q, atol=1e-12)
