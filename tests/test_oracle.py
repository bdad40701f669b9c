"""Pins for the CPU oracle: each check ties it to something other than itself
(closed forms, LAPACK special cases, QR uniqueness, the paper's printed
accuracy), chosen so that a dropped term, sign or transposition fails."""
import json
import math
import os

import numpy as np
import pytest

from oracle import blr_qr as O
from oracle import dense_qr as D
from paper_2208_06194_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiles_of(a, b):
    return lambda i, j: a[i * b:(i + 1) * b, j * b:(j + 1) * b]


def explicit_householder_product(ys, taus):
    """H_0 H_1 ... with H_j = I - tau_j y_j y_j^T (closed form of Eq. 3)."""
    m = ys.shape[0]
    q = np.eye(m)
    for j in range(ys.shape[1]):
        y = ys[:, j]
        q = q @ (np.eye(m) - taus[j] * np.outer(y, y))
    return q


# ---------------------------------------------------------------- reflector

@pytest.mark.parametrize("x", [[3.0, 4.0], [-3.0, 4.0, 0.0], [0.0, 1.0, 2.0], [2.0, 0.0, 0.0]])
def test_reflector_maps_to_beta_e1(x):
    x = np.array(x)
    beta, tau, v = D.reflector(x)
    h = np.eye(len(x)) - tau * np.outer(v, v)
    e = np.zeros_like(x)
    e[0] = beta
    assert np.allclose(h @ x, e, atol=1e-14)
    assert abs(abs(beta) - np.linalg.norm(x)) < 1e-14
    assert np.allclose(h @ h.T, np.eye(len(x)), atol=1e-14)
    if np.linalg.norm(x[1:]) == 0:
        assert tau == 0.0 and beta == x[0]
    else:
        assert 1.0 <= tau <= 2.0
        assert beta * x[0] <= 0.0  # beta = -sign(alpha) ||x||


def test_dense_qr_matches_lapack():
    """Textbook QR == LAPACK dgeqrf (same sign convention), R to 1e-13."""
    a = np.random.default_rng(1).standard_normal((40, 17))
    r, refl = D.householder_qr(a)
    r_lapack = np.linalg.qr(a, mode="r")
    assert np.allclose(r, r_lapack, atol=1e-13 * np.abs(r).max())
    q1 = D.thin_q(refl, 40, 17)
    assert np.allclose(q1 @ r, a, atol=1e-13)
    assert np.allclose(q1.T @ q1, np.eye(17), atol=1e-14)


# ---------------------------------------------------------------- tile kernels

def test_geqrt_compact_wy_equals_product_of_reflectors():
    a = np.random.default_rng(2).standard_normal((12, 12))
    r, y, t = O.geqrt(a)
    assert np.allclose(np.tril(y), y) and np.allclose(np.diag(y), 1.0)
    assert np.allclose(np.triu(t), t)
    q = np.eye(12) - y @ t @ y.T
    assert np.allclose(q, explicit_householder_product(y, np.diag(t)), atol=1e-14)
    assert np.allclose(q @ r, a, atol=1e-13)
    assert np.allclose(r, np.linalg.qr(a, mode="r"), atol=1e-13)


@pytest.mark.parametrize("rows", [0, 1, 3, 8])
def test_tsqrt_update_qr(rows):
    rng = np.random.default_rng(3 + rows)
    b = 8
    r0 = np.triu(rng.standard_normal((b, b)))
    bv = rng.standard_normal((rows, b))
    r1, y, t = O.tsqrt(r0, bv)
    yy = np.vstack([np.eye(b), y])
    q = np.eye(b + rows) - yy @ t @ yy.T
    assert np.allclose(q.T @ q, np.eye(b + rows), atol=1e-14)
    stacked = np.vstack([r0, bv])
    target = np.vstack([r1, np.zeros((rows, b))])
    assert np.allclose(q.T @ stacked, target, atol=1e-13)
    assert np.allclose(np.triu(r1), r1)
    # uniqueness of R up to row signs (Trefethen & Bau, Thm 7.2)
    assert np.allclose(D.sign_normalize(r1),
                       D.sign_normalize(np.linalg.qr(stacked, mode="r")), atol=1e-13)
    assert np.allclose(q, explicit_householder_product(yy, np.diag(t)), atol=1e-14)


def test_lifted_reflector_orthogonal_iff_u_orthonormal():
    """Eq. 21: I - [I; U Y] T [I; U Y]^T is orthogonal when U^T U = I."""
    rng = np.random.default_rng(4)
    b, r = 10, 3
    r0 = np.triu(rng.standard_normal((b, b)))
    vt = rng.standard_normal((r, b))
    _, y, t = O.tsqrt(r0, vt)
    u, _ = np.linalg.qr(rng.standard_normal((b, r)))
    for scale, ok in [(1.0, True), (1.3, False)]:
        yt = np.vstack([np.eye(b), scale * u @ y])
        q = np.eye(2 * b) - yt @ t @ yt.T
        err = np.linalg.norm(q.T @ q - np.eye(2 * b))
        assert (err < 1e-13) == ok


def test_larfb_is_qt_times_c():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((9, 9))
    _, y, t = O.geqrt(a)
    c = rng.standard_normal((9, 4))
    qt = (np.eye(9) - y @ t @ y.T).T
    assert np.allclose(O.larfb(y, t, c), qt @ c, atol=1e-13)


def _rand_tile(rng, b, kind, r):
    if kind == "D":
        return O.dense_tile(rng.standard_normal((b, b)))
    u, _ = np.linalg.qr(rng.standard_normal((b, r)))
    return O.lr_tile(u, rng.standard_normal((b, r)))


@pytest.mark.parametrize("ykind", ["L", "D"])
@pytest.mark.parametrize("rkind", ["L", "D"])
@pytest.mark.parametrize("akind", ["L", "D"])
def test_tpmqrt_equals_dense_trapezoidal_reflector(ykind, rkind, akind):
    rng = np.random.default_rng(["LLL", "LLD", "LDL", "LDD", "DLL", "DLD", "DDL", "DDD"].index(ykind + rkind + akind))
    b, r = 16, 3
    rkk = np.triu(rng.standard_normal((b, b)))
    aik = _rand_tile(rng, b, ykind, r)
    bv = aik.v.T if ykind == "L" else aik.d
    _, yik, t = O.tsqrt(rkk, bv)
    ytile = O.lr_tile(aik.u, yik.T) if ykind == "L" else O.dense_tile(yik)
    rkj = _rand_tile(rng, b, rkind, 2)
    aij = _rand_tile(rng, b, akind, 4)
    yt = ytile.dense()
    full = np.vstack([np.eye(b), yt])
    qt = (np.eye(2 * b) - full @ t @ full.T).T
    want = qt @ np.vstack([rkj.dense(), aij.dense()])
    for eps, tol in [(1e-15, 1e-12), (1e-6, 3e-5)]:
        r_new, a_new = O.tpmqrt(ytile, t, rkj, aij, eps, b // 2)
        got = np.vstack([r_new.dense(), a_new.dense()])
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
        if rkind == "L" and (ykind == "L" or akind == "L"):
            assert r_new.kind == "L" or r_new.rank == -1
        if rkind == "D":
            assert r_new.kind == "D"


# ---------------------------------------------------------------- BLR arithmetic

def test_truncation_rank_closed_form():
    s = np.array([1.0, 1e-3, 1e-6, 1e-9])
    # tails: r=1 -> sqrt(1e-6+1e-12+1e-18) ~ 1e-3
    total = math.sqrt(np.sum(s ** 2))
    assert O.truncation_rank(s, 2e-3 / total) == 1
    assert O.truncation_rank(s, 0.5e-3 / total) == 2
    assert O.truncation_rank(s, 0.0) == 4
    assert O.truncation_rank(np.zeros(3), 1e-8) == 0
    assert O.truncation_rank(s, 10.0) == 0


def test_rounded_addition_bound_orthonormal_and_rank():
    rng = np.random.default_rng(6)
    b = 30
    # A + B has exactly the singular values sig (planted), so the rank is known
    uo, _ = np.linalg.qr(rng.standard_normal((b, 6)))
    vo, _ = np.linalg.qr(rng.standard_normal((b, 6)))
    sig = np.array([5.0, 2.0, 1.0, 1e-4, 1e-9, 1e-12])
    c = uo @ np.diag(sig) @ vo.T
    ua, _ = np.linalg.qr(rng.standard_normal((b, 4)))
    va = rng.standard_normal((b, 4))
    # B = C - A written as low rank (U_B = [uo, ua], V_B = [vo sig, -va])
    ub = np.hstack([uo, ua])
    vb = np.hstack([vo * sig, -va])
    for eps, want_rank in [(1e-2, 3), (1e-6, 4), (1e-10, 5), (1e-14, 6)]:
        out = O.rounded_addition(ua, va, ub, vb, eps, b // 2)
        assert out.kind == "L" and out.rank == want_rank
        err = np.linalg.norm(out.dense() - c)
        assert err <= eps * np.linalg.norm(c) * (1 + 1e-6) + 1e-13
        assert np.allclose(out.u.T @ out.u, np.eye(want_rank), atol=1e-13)


def test_rounded_addition_over_cap_goes_dense():
    rng = np.random.default_rng(7)
    b = 8
    ua, va = rng.standard_normal((b, 4)), rng.standard_normal((b, 4))
    ub, vb = rng.standard_normal((b, 4)), rng.standard_normal((b, 4))
    out = O.rounded_addition(ua, va, ub, vb, 0.0, b // 2)
    assert out.kind == "D"
    assert np.allclose(out.d, ua @ va.T + ub @ vb.T, atol=1e-13)


def test_dense_threshold_below_half_b():
    """A dense threshold below b/2 (Section 3.1's dense fallback with a lower
    threshold): a sum or a tile whose rank exceeds it is stored dense (the
    exact sum / the tile itself), one at the threshold stays low-rank; the
    factorization keeps every low-rank tile at or below the threshold and
    still equals the textbook dense QR (QR uniqueness)."""
    rng = np.random.default_rng(17)
    b = 16
    uo, _ = np.linalg.qr(rng.standard_normal((b, 5)))
    vo = rng.standard_normal((b, 5))
    c = uo @ vo.T                                  # exact rank 5
    for cap, kind in [(4, "D"), (5, "L"), (8, "L")]:
        out = O.rounded_addition(uo[:, :3], vo[:, :3], uo[:, 3:], vo[:, 3:], 1e-12, cap)
        assert out.kind == kind, cap
        assert np.linalg.norm(out.dense() - c) <= 1e-12 * np.linalg.norm(c)
        if kind == "L":
            assert out.rank == 5
        t = O.compress_qrcp(c, 1e-12, cap)
        assert t.kind == kind, cap
        if kind == "D":
            assert np.array_equal(t.d, c)
        else:
            assert t.rank == 5
    # the matrix carries its threshold; 0 and values above b/2 mean b/2
    assert O.BLRMatrix(1, 1, 16, [], 3).cap == 3
    assert O.BLRMatrix(1, 1, 16, [], 0).cap == 8
    assert O.BLRMatrix(1, 1, 16, [], 9).cap == 8
    # compression at threshold 2 of exact ranks 1..3: rank-3 tiles dense
    m, n, b = 96, 48, 8
    a = np.zeros((m, n))
    ranks = {}
    for j in range(n // b):
        for i in range(m // b):
            k = b if i == j else 1 + (i + 2 * j) % 3
            a[i * b:(i + 1) * b, j * b:(j + 1) * b] = rng.standard_normal((b, k)) @ rng.standard_normal((k, b))
            ranks[i, j] = k
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14, dense_rank=2)
    assert blr.cap == 2
    for (i, j), k in ranks.items():
        t = blr.tiles[i][j]
        assert (t.kind == "D") == (i == j or k > 2), (i, j)
        if t.kind == "L":
            assert t.rank == k
    f = O.blr_qr(blr, 1e-15)
    rk = f.ranks()
    assert rk.max() <= 2
    assert (rk == -1).sum() > (blr.ranks() == -1).sum()       # sums above the threshold went dense
    r_dense = np.linalg.qr(a, mode="r")
    assert np.linalg.norm(D.sign_normalize(f.r_dense()) - D.sign_normalize(r_dense)) <= 1e-12 * np.linalg.norm(r_dense)
    assert O.residual(f, a) < 1e-13


def test_strong_admissibility_box_distance():
    """Strong admissibility (Section 3.1, eta) on boxes computed by hand: a
    tile is near when the gap between its clusters' bounding boxes is below
    eta times the larger box diameter; a larger eta keeps more tiles dense;
    eta = 0 keeps none."""
    b = 2
    # row clusters: box [0,1]^3 (diameter sqrt 3) and box [0,3] x [0,0] x [0,0] (diameter 3)
    x = np.array([[0.0, 1.0, 0.0, 3.0],
                  [0.0, 1.0, 0.0, 0.0],
                  [0.0, 1.0, 0.0, 0.0]])
    # column cluster: box [2,2.5] x [0,0] x [0,0] (diameter 0.5)
    y = np.array([[2.0, 2.5],
                  [0.0, 0.0],
                  [0.0, 0.0]])
    # gaps: cluster 0 -> (1, 0, 0): distance 1, larger diameter sqrt 3;
    #       cluster 1 -> overlapping boxes: distance 0, larger diameter 3
    for eta, want in [(0.0, [False, False]), (0.5, [False, True]), (1.0 / math.sqrt(3) - 1e-9, [False, True]),
                      (1.0 / math.sqrt(3) + 1e-9, [True, True]), (2.0, [True, True])]:
        near = O.strong_admissibility(x, y, b, eta)
        assert near.shape == (2, 1)
        assert list(near[:, 0]) == want, eta
    # monotone in eta on a kernel workload; diagonal-distance ordering kept
    pr = W.kernel_problem("yukawa3d", 1024, 512, 64, 5, 6)
    counts = [int(O.strong_admissibility(pr.x, pr.y, 64, eta).sum()) for eta in (0.0, 0.3, 1.0, 3.0)]
    assert counts[0] == 0 and counts == sorted(counts) and counts[-1] > counts[1]
    # compress() keeps the near tiles dense, compresses the rest
    near = O.strong_admissibility(pr.x, pr.y, 64, 1.0)
    blr = O.compress(pr.tile, 16, 8, 64, eps=1e-3, inadmissible=near)
    rk = blr.ranks()
    assert (rk[near] == -1).all()
    weak = O.compress(pr.tile, 16, 8, 64, eps=1e-3).ranks()
    far = ~near & ~np.eye(16, 8, dtype=bool)
    assert np.array_equal(rk[far], weak[far])
    assert (weak[near & ~np.eye(16, 8, dtype=bool)] >= 0).any()    # near tiles that weak admissibility compresses


def test_op3_op4_products():
    rng = np.random.default_rng(8)
    x = O.lr_tile(rng.standard_normal((7, 2)), rng.standard_normal((7, 2)))
    y = O.lr_tile(rng.standard_normal((7, 3)), rng.standard_normal((7, 3)))
    d = O.dense_tile(rng.standard_normal((7, 7)))
    for p, q in [(x, y), (x, d), (d, y), (d, d)]:
        prod = O.mul(p, q)
        assert np.allclose(prod.dense(), p.dense() @ q.dense(), atol=1e-12)
    assert O.mul(x, y).rank == 2  # OP4 keeps U_A (rank of the left factor)


def test_compress_qrcp_tolerance_and_exact_rank():
    rng = np.random.default_rng(9)
    b = 32
    a = rng.standard_normal((b, 5)) @ rng.standard_normal((5, b))
    t = O.compress_qrcp(a, 1e-12, b // 2)
    assert t.kind == "L" and t.rank == 5
    assert np.allclose(t.u.T @ t.u, np.eye(5), atol=1e-14)
    assert np.linalg.norm(t.dense() - a) <= 1e-12 * np.linalg.norm(a)
    # smooth kernel tile: tolerance met, rank >= the SVD's optimal rank
    pr = W.kernel_problem("yukawa3d", 256, 256, 64, 11, 12)
    tile = pr.tile(0, 3)
    for eps in [1e-4, 1e-8]:
        t = O.compress_qrcp(tile, eps, 32)
        assert np.linalg.norm(t.dense() - tile) <= eps * np.linalg.norm(tile)
        s = np.linalg.svd(tile, compute_uv=False)
        assert t.kind == "D" or t.rank >= O.truncation_rank(s, eps)
    # pivots take the largest remaining column: on the smooth tile the rank
    # stays within a few of the SVD's optimum (a pivot on a small column
    # inflates it past the dense threshold)
    t = O.compress_qrcp(tile, 1e-4, 32)
    s = np.linalg.svd(tile, compute_uv=False)
    assert t.kind == "L" and t.rank <= O.truncation_rank(s, 1e-4) + 4
    # orthogonal columns of norms 10^-l in shuffled positions among zero
    # columns: the pivoted QR takes them largest first, so its truncation is
    # the SVD's exactly (same rank, same leading directions)
    sig = 10.0 ** -np.arange(12.0)
    uo, _ = np.linalg.qr(rng.standard_normal((b, 12)))
    cols = rng.permutation(b)[:12]
    a = np.zeros((b, b))
    a[:, cols] = uo * sig
    for eps in [1e-3, 1e-7, 1e-11]:
        t = O.compress_qrcp(a, eps, b // 2)
        r = O.truncation_rank(sig, eps)
        assert t.kind == "L" and t.rank == r
        assert np.allclose(np.abs(t.u), np.abs(uo[:, :r]), atol=1e-12)
    # full-rank random tile needs rank > b/2 -> dense, unchanged
    g = rng.standard_normal((b, b))
    t = O.compress_qrcp(g, 1e-8, b // 2)
    assert t.kind == "D" and np.array_equal(t.d, g)
    z = O.compress_qrcp(np.zeros((b, b)), 1e-8, b // 2)
    assert z.kind == "L" and z.rank == 0


# ---------------------------------------------------------------- Algorithm 4

@pytest.mark.parametrize("m,n,b", [(32, 16, 4), (64, 32, 8)])
def test_full_rank_blr_equals_dense_qr(m, n, b):
    """Dense tiles everywhere: tiled QR == textbook QR up to row signs."""
    a = np.random.default_rng(m).standard_normal((m, n))
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=0.0)
    assert (blr.ranks() == -1).all()
    f = O.blr_qr(blr, 0.0)
    r_dense, _ = D.householder_qr(a)
    r = f.r_dense()
    assert np.abs(np.abs(np.diag(r)) - np.abs(np.diag(r_dense))).max() < 1e-13 * np.abs(r).max()
    assert np.allclose(D.sign_normalize(r), D.sign_normalize(r_dense), atol=1e-13 * np.abs(r).max())


@pytest.mark.parametrize("m,n,b,k", [(128, 64, 16, 2), (96, 48, 8, 1)])
def test_exact_low_rank_blr_equals_dense_qr(m, n, b, k):
    """Exact rank-k off-diagonal tiles: the low-rank path reproduces dense QR."""
    a = W.random_blr_dense(m, n, b, k, seed=m + k)
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    ranks = blr.ranks()
    assert (ranks[~np.eye(m // b, n // b, dtype=bool)] == k).all()
    f = O.blr_qr(blr, 1e-15)
    r = f.r_dense()
    r_dense = np.linalg.qr(a, mode="r")
    assert np.linalg.norm(D.sign_normalize(r) - D.sign_normalize(r_dense)) <= 1e-12 * np.linalg.norm(r)
    assert O.residual(f, a) < 1e-13
    assert O.orthogonality(f) < 1e-13


def test_apply_q_roundtrip_and_qt_a_is_r():
    a = W.random_blr_dense(96, 48, 8, 2, seed=3)
    blr = O.compress(tiles_of(a, 8), 12, 6, 8, eps=1e-14)
    f = O.blr_qr(blr, 1e-15)
    c = np.random.default_rng(0).standard_normal((96, 3))
    assert np.allclose(O.apply_qt(f, O.apply_q(f, c)), c, atol=1e-13)
    qta = O.apply_qt(f, a)
    assert np.allclose(qta[:48], f.r_dense(), atol=1e-12 * np.abs(a).max())
    assert np.abs(qta[48:]).max() < 1e-12 * np.abs(a).max()


def test_metrics_measure_planted_errors():
    """Res and Orth (Section 5) on errors of known size: against (1 + d) A an
    exact factorization has Res = d / (1 + d); a Q whose every column is
    scaled by (1 + d) (the thin Q of the exact factor times (1 + d)) has
    Q^T Q - I = ((1 + d)^2 - 1) I, so Orth = (2d + d^2) sqrt(n) / sqrt(n)."""
    a = W.random_blr_dense(96, 48, 8, 2, seed=3)
    blr = O.compress(tiles_of(a, 8), 12, 6, 8, eps=1e-14)
    f = O.blr_qr(blr, 1e-15)
    for d in (1e-3, 1e-6):
        assert O.residual(f, a * (1 + d)) == pytest.approx(d / (1 + d), rel=1e-6)
    q1 = O.thin_q(f)
    assert q1.shape == (96, 48)
    for d in (1e-3, 1e-6):
        scaled = q1 * (1 + d)
        orth = np.linalg.norm(scaled.T @ scaled - np.eye(48)) / math.sqrt(48)
        assert orth == pytest.approx(2 * d + d * d, rel=1e-6)
    assert O.orthogonality(f) < 1e-13
    # thin_q is Q [I; 0]: Q^T applied to it gives back [I; 0]
    e = np.zeros((96, 48))
    e[:48] = np.eye(48)
    assert np.allclose(O.apply_qt(f, q1), e, atol=1e-13)


def test_lstsq_matches_library_and_refinement():
    a = W.random_blr_dense(96, 48, 8, 2, seed=4)
    blr = O.compress(tiles_of(a, 8), 12, 6, 8, eps=1e-14)
    f = O.blr_qr(blr, 1e-15)
    bm = W.gaussian_rhs(96, 2, 5)
    x = O.lstsq(f, bm)
    x_ref = np.linalg.lstsq(a, bm, rcond=None)[0]
    assert np.allclose(x, x_ref, atol=1e-10 * np.abs(x_ref).max())
    x2 = O.lstsq(f, bm, blr, refine_steps=1)
    g1 = np.linalg.norm(a.T @ (bm - a @ x))
    g2 = np.linalg.norm(a.T @ (bm - a @ x2))
    assert g2 <= max(g1, 1e-12 * np.linalg.norm(a) * np.linalg.norm(bm))


def test_inv1d_invariants():
    """2048 x 1024, b = 128, fixed rank 8: Res against A~ at 1e-12 level,
    Orth at round-off, R R^T structure, and R^T R = A~^T A~."""
    pr = W.inv1d_2048x1024()
    blr = O.compress(pr.tile, 16, 8, 128, fixed_rank=8)
    f = O.blr_qr(blr, 1e-14)
    at = blr.dense()
    assert O.residual(f, at) < 1e-12
    assert O.orthogonality(f) < 1e-13
    r = f.r_dense()
    assert np.allclose(r, np.triu(r))
    gram = at.T @ at
    assert np.linalg.norm(r.T @ r - gram) < 1e-13 * np.linalg.norm(gram)


@pytest.mark.slow
def test_paper_random_accuracy_table():
    """Section 5.1 printed accuracy (tiled Householder) at 2048 x 1024."""
    with open(os.path.join(GOLDEN, "table_res_acc_random.json")) as fh:
        row = json.load(fh)["rows"][0]
    m, n, b, k, eps = row["m"], row["n"], row["b"], row["k"], row["eps"]
    a = W.random_blr_dense(m, n, b, k, seed=7)
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=eps)
    f = O.blr_qr(blr, eps)
    res = O.residual(f, a)
    orth = O.orthogonality(f)
    assert res <= 10 * row["res"]
    assert orth <= row["orth"]


# ---------------------------------------------------------------- inputs

def test_kernel_entries_closed_form():
    x = np.array([[0.0, 0.5]])
    y = np.array([[0.25]])
    a = W.kernel_entries("inv1d", x, y)
    assert np.allclose(a[:, 0], [1 / (0.25 + 1e-3), 1 / (0.25 + 1e-3)])
    x3 = np.array([[0.0], [0.0], [0.0]])
    y3 = np.array([[0.3], [0.4], [0.0]])
    assert np.isclose(W.kernel_entries("yukawa3d", x3, y3)[0, 0], math.exp(-0.5) / 0.501)
    assert np.isclose(W.kernel_entries("laplace3d", x3, y3)[0, 0], 1 / 0.501)


def test_rcb_order_leaves_and_boxes():
    pts = np.random.default_rng(0).random((3, 6 * 8))
    perm = W.rcb_order(pts, 8)
    assert sorted(perm.tolist()) == list(range(48))
    # first split: longest side, 3 of 6 leaves on the left
    dim = int(np.argmax(pts.max(1) - pts.min(1)))
    left = pts[dim, perm[:24]]
    right = pts[dim, perm[24:]]
    assert left.max() <= right.min()
    # every leaf keeps ascending original index
    for leaf in range(6):
        ids = perm[leaf * 8:(leaf + 1) * 8]
        assert (np.diff(ids) > 0).all()


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_rcb_odd_leaf_count_and_anisotropic_box(seed):
    """5 leaves: the first split sends ceil(5/2) = 3 leaves left, along the
    box's longest side (x: extents 3, 2, 0.25); the left 3 leaves then split
    2 + 1 along their own longest side (y for most draws)."""
    pts = np.random.default_rng(seed).random((3, 5 * 4)) * np.array([[3.0], [2.0], [0.25]])
    perm = W.rcb_order(pts, 4)
    assert sorted(perm.tolist()) == list(range(20))
    assert pts[0, perm[:12]].max() <= pts[0, perm[12:]].min()
    sub = pts[:, perm[:12]]
    d2 = int(np.argmax(sub.max(1) - sub.min(1)))
    assert pts[d2, perm[:8]].max() <= pts[d2, perm[8:12]].min()


def test_ill_conditioned_scale():
    d = W.ill_conditioned_scale(11)
    assert d[0] == 1.0 and np.isclose(d[-1], 1e-10)
    assert np.allclose(d[1:] / d[:-1], 10 ** (-1.0))


def test_column_scaling_is_a_right_diagonal_factor():
    """The ill-conditioned variant is A D with D = diag(d) acting on columns:
    every block is the unscaled block times d of its columns, and the dense
    QR of A D has R(A D) = R(A) D up to row signs (Householder QR commutes
    with a positive column scaling in exact arithmetic)."""
    base = W.kernel_problem("yukawa3d", 48, 24, 8, 31, 32)
    ill = W.kernel_problem("yukawa3d", 48, 24, 8, 31, 32, ill_conditioned=True)
    d = W.ill_conditioned_scale(24)
    assert np.allclose(ill.block(8, 24, 0, 8), base.block(8, 24, 0, 8) * d[None, :8], rtol=1e-15)
    assert np.allclose(ill.block(0, 24, 0, 24), base.block(0, 24, 0, 24) * d[None, :], rtol=1e-15)
    a, ad = base.dense(), ill.dense()
    r_a = D.sign_normalize(np.linalg.qr(a, mode="r"))
    r_ad = D.sign_normalize(np.linalg.qr(ad, mode="r"))
    # column j of R(A) D: compare column by column relative to its own size
    want = r_a * d[None, :]
    for j in range(24):
        assert np.linalg.norm(r_ad[:, j] - want[:, j]) <= 1e-8 * np.linalg.norm(want[:, j])


# ---------------------------------------------------------------- blocked variant (Section 3.3)

@pytest.mark.parametrize("m,n,b", [(32, 16, 4), (48, 24, 8)])
def test_blocked_full_rank_equals_dense_qr(m, n, b):
    """Dense tiles everywhere: the block-column QR is the textbook QR of the
    whole matrix (QR uniqueness up to row signs)."""
    a = np.random.default_rng(m + 1).standard_normal((m, n))
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=0.0)
    f = O.blr_qr_blocked(blr, 0.0)
    r_dense, _ = D.householder_qr(a)
    assert np.allclose(D.sign_normalize(f.r_dense()), D.sign_normalize(r_dense), atol=1e-13 * np.abs(r_dense).max())


@pytest.mark.parametrize("m,n,b,k", [(128, 64, 16, 2), (96, 48, 8, 1)])
def test_blocked_exact_low_rank_matches_dense_and_tiled(m, n, b, k):
    """Exact rank-k tiles: the blocked variant gives the dense QR's R (up to
    row signs), the same R as the tiled Algorithm 4, an orthogonal Q and
    Q^T A = [R; 0]."""
    a = W.random_blr_dense(m, n, b, k, seed=m + 2 * k)
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    fb = O.blr_qr_blocked(blr, 1e-15)
    ft = O.blr_qr(blr, 1e-15)
    rb = D.sign_normalize(fb.r_dense())
    assert np.linalg.norm(rb - D.sign_normalize(np.linalg.qr(a, mode="r"))) <= 1e-12 * np.linalg.norm(rb)
    assert np.linalg.norm(rb - D.sign_normalize(ft.r_dense())) <= 1e-12 * np.linalg.norm(rb)
    e = np.zeros((m, n))
    e[:n] = np.eye(n)
    q1 = O.blocked_apply_q(fb, e)
    assert np.linalg.norm(q1.T @ q1 - np.eye(n)) / np.sqrt(n) < 1e-13
    qta = O.blocked_apply_qt(fb, a)
    assert np.linalg.norm(qta[:n] - fb.r_dense()) <= 1e-12 * np.linalg.norm(a)
    assert np.linalg.norm(qta[n:]) <= 1e-12 * np.linalg.norm(a)


def test_blocked_tails_keep_the_blr_structure():
    """Y~_ik = A^U_ik Y_ik (Section 3.3.1): low-rank with A_ik's own U where
    A_ik is low-rank (checked on the first block column, before any update
    changes the tiles; later ones may have become dense through rank growth),
    an orthonormal U wherever it is low-rank, and a unit lower triangular
    tail in the diagonal block."""
    m, n, b, k = 64, 32, 8, 2
    a = W.random_blr_dense(m, n, b, k, seed=5)
    blr = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    f = O.blr_qr_blocked(blr, 1e-15)
    for kk in range(n // b):
        for off, yt in enumerate(f.y[kk]):
            i = kk + off
            if i == kk:
                assert yt.kind == "D" and np.allclose(np.triu(yt.d), np.eye(b))
                continue
            if kk == 0:                       # the input's low-rank tiles
                assert yt.kind == "L" and np.array_equal(yt.u, blr.tiles[i][0].u)
            if yt.kind == "L":                # later columns: tiles the updates left low-rank
                assert np.allclose(yt.u.T @ yt.u, np.eye(yt.u.shape[1]), atol=1e-12)
                assert yt.v.shape == (b, yt.u.shape[1])


def test_blocked_with_truncation_meets_the_tolerance():
    """A kernel matrix compressed at 1e-8 and factored with rounded
    additions at 1e-8: Res against A~ at the tolerance level, Q orthogonal."""
    pr = W.kernel_problem("yukawa3d", 256, 128, 32, 71, 72)
    blr = O.compress(pr.tile, 8, 4, 32, eps=1e-8)
    f = O.blr_qr_blocked(blr, 1e-8)
    at = blr.dense()
    e = np.zeros((256, 128))
    e[:128] = np.eye(128)
    q1 = O.blocked_apply_q(f, e)
    assert np.linalg.norm(q1 @ f.r_dense() - at) <= 10 * 1e-8 * np.linalg.norm(at)
    assert np.linalg.norm(q1.T @ q1 - np.eye(128)) / np.sqrt(128) < 1e-12
