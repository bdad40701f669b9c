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
    # reading 7: applying the inner blocks one after another (the stored
    # T_J, nb reflectors each) is the same Q
    q_inner = np.eye(2 * b)
    for j0 in range(0, b, nb):
        vj = full[:, j0:j0 + nb]
        q_inner = q_inner @ (np.eye(2 * b) - vj @ t[j0:j0 + nb, j0:j0 + nb] @ vj.T)
    assert np.allclose(q_inner, q, atol=1e-12)


# ---------------------------------------------------------------- reading 9

def _rounded_addition_qrcp(ua, va, ub, vb, eps):
    """Reading 9: Algorithm 6 with the s x s core R_U R_V^T truncated by a
    column-pivoted QR (stop at the first r whose trailing block has Frobenius
    norm <= eps times the core's) instead of its SVD."""
    qu, ru = np.linalg.qr(np.hstack([ua, ub]))
    qv, rv = np.linalg.qr(np.hstack([va, vb]))
    c = ru @ rv.T
    t = O.compress_qrcp(c, eps, c.shape[1])     # C ~ Q_C R_C P^T: U = Q_C, V = P R_C^T
    if t.kind == "D":
        return qu @ c @ qv.T, c.shape[1]
    return qu @ t.u @ (qv @ t.v).T, t.rank


@pytest.mark.parametrize("decay", [0.5, 0.1])
def test_pivoted_qr_core_truncation_meets_the_bound(decay):
    """The pivoted-QR truncation of the core meets Algorithm 6's Frobenius
    bound (||C - C_r||_F <= eps ||C||_F, exact because Q_U and Q_V are
    orthonormal) with a rank at or a few above the SVD's."""
    rng = np.random.default_rng(int(decay * 10))
    b, ra, rb = 64, 10, 12
    sig = decay ** np.arange(ra + rb)
    x, _ = np.linalg.qr(rng.standard_normal((b, ra + rb)))
    z, _ = np.linalg.qr(rng.standard_normal((b, ra + rb)))
    total = x @ np.diag(sig) @ z.T                    # A + B with a known spectrum
    ua, _ = np.linalg.qr(rng.standard_normal((b, ra)))
    va = rng.standard_normal((b, ra))
    ub = np.hstack([x, ua])                             # B = total - A as a rank-(ra+rb+ra) product
    vb = np.hstack([z * sig, -va])
    for eps in (1e-2, 1e-5, 1e-9):
        got, r = _rounded_addition_qrcp(ua, va, ub, vb, eps)
        assert np.linalg.norm(got - total) <= eps * np.linalg.norm(total) * (1 + 1e-8) + 1e-14
        r_svd = O.truncation_rank(sig, eps)
        assert r_svd <= r <= r_svd + 3, (eps, r, r_svd)
