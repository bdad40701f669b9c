"""GPU parity: the CUDA path against the CPU oracle on the same seeded inputs.

Elementwise parity needs a well-determined R, so the exact-input cases use
the paper's random BLR matrices (Section 5.1 generator: dense N(0,1)
diagonal tiles, rank-k off-diagonal tiles), which are well conditioned.
Both sides factor the identical A~ (the oracle's compression, imported
through blr_matrix_import).  Tolerances: with kappa(A~) = O(10-100) and
recompression at 1e-14, R, Y~ and Q agree to 1e-11 relative; Orth is the
FP64 target 1e-12; Res is checked at 10x the recompression tolerance.
"""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import lib_r_dense, lib_tile, lib_to_oracle, lib_y_dense, oracle_to_lib, tiles_of

pytestmark = pytest.mark.gpu


def _mixed_blr(m, n, b, seed, dense_offdiag=(), zero_tiles=()):
    """Random BLR with ranks 1..3, some dense off-diagonal and zero tiles."""
    rng = np.random.default_rng(seed)
    p, q = m // b, n // b
    a = np.zeros((m, n))
    for j in range(q):
        for i in range(p):
            if (i, j) in zero_tiles:
                continue
            if i == j or (i, j) in dense_offdiag:
                t = rng.standard_normal((b, b))
            else:
                k = 1 + (i + 2 * j) % 3
                t = rng.standard_normal((b, k)) @ rng.standard_normal((b, k)).T
            a[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
    return a


def _factor_both(lib, a, b, eps=1e-14, rec=1e-14):
    m, n = a.shape
    p, q = m // b, n // b
    ref = O.compress(tiles_of(a, b), p, q, b, eps=eps)
    ranks, tiles = oracle_to_lib(ref)
    mat = lib.blr_matrix_import(m, n, b, ranks, tiles)
    fac = lib.blr_qr(mat, lib.blr_opts_default(b=b, tol=eps, rec_tol=rec))
    fo = O.blr_qr(ref, rec)
    return ref, fac, fo


CASES = [
    (256, 128, 32, 1, (), ()),
    (224, 96, 32, 2, ((3, 0), (5, 2)), ((4, 1),)),
    (672, 288, 96, 3, ((6, 1),), ((2, 0),)),          # b = 96: ragged 64-column chunks
    (512, 512, 64, 4, ((3, 1),), ()),                 # square: no TSQRT below the last diagonal
    (320, 64, 64, 5, (), ()),                         # single block column
]


@pytest.mark.parametrize("m,n,b,seed,dense,zero", CASES)
def test_exact_input_factor_parity(lib, m, n, b, seed, dense, zero):
    a = _mixed_blr(m, n, b, seed, dense, zero)
    ref, fac, fo = _factor_both(lib, a, b)
    p, q = m // b, n // b
    rk, tl = lib.blr_matrix_export(fac)
    # ranks after the factorization: integer, bit-exact
    ro = np.array([[fo.tiles[i][j].rank for j in range(q)] for i in range(p)])
    rg = rk.reshape(q, p).T
    assert np.array_equal(rg, ro), f"ranks differ:\n{rg}\n{ro}"
    # R elementwise
    r_g = lib_r_dense(rk, tl, p, q, b)
    r_o = fo.r_dense()
    assert np.linalg.norm(r_g - r_o) <= 1e-11 * np.linalg.norm(r_o)
    # reflectors: Y_kk and Y~_ik elementwise
    for k in range(q):
        yg = lib_y_dense(rk, tl, p, b, k, k)
        assert np.allclose(yg, fo.y_diag(k), atol=1e-11 * max(1.0, np.abs(yg).max()))
        for i in range(k + 1, p):
            yg = lib_y_dense(rk, tl, p, b, i, k)
            yo = fo.y_dense(i, k)
            assert np.linalg.norm(yg - yo) <= 1e-11 * max(1.0, np.linalg.norm(yo)), (i, k)
    fac.destroy()


@pytest.mark.parametrize("m,n,b,seed,dense,zero", CASES[:3])
def test_q_application_parity(lib, m, n, b, seed, dense, zero):
    import torch
    a = _mixed_blr(m, n, b, seed, dense, zero)
    ref, fac, fo = _factor_both(lib, a, b)
    c = np.random.default_rng(seed + 100).standard_normal((m, 5))   # 5: ragged column group
    for trans in (0, 1):
        ct = lib.to_fortran(torch.from_numpy(c))
        lib.blr_apply_qt(fac, ct, trans=trans)
        got = ct.cpu().numpy()
        want = O.apply_qt(fo, c) if trans == 0 else O.apply_q(fo, c)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(c)
    fac.destroy()


@pytest.mark.parametrize("m,n,b,nrhs", [(1024, 512, 128, 700), (2048, 1024, 512, 150), (512, 512, 64, 33)])
def test_q_application_over_several_column_groups(lib, m, n, b, nrhs):
    """The pipelined Q application splits each TSQRT's b/32 reflector
    blocks over as many CTAs and runs 16 right-hand sides per group, as many
    groups per launch as the SMs hold at once (one CTA per SM).  700 columns
    at b = 128 (44 groups of 4 CTAs) and 150 at b = 512 (10 groups of 16)
    take two launches; the square case has no update QR below the last
    diagonal tile and a ragged last group.  Q^T B and Q B against the
    oracle, low-rank, dense and zero reflector blocks mixed."""
    import torch
    p, q = m // b, n // b
    a = _mixed_blr(m, n, b, 11 + b, ((p - 1, 0), (2, 1)), ((p - 2, 0),))
    ref, fac, fo = _factor_both(lib, a, b)
    c = np.random.default_rng(b + nrhs).standard_normal((m, nrhs))
    for trans in (0, 1):
        ct = lib.to_fortran(torch.from_numpy(c))
        lib.blr_apply_qt(fac, ct, trans=trans)
        got = ct.cpu().numpy()
        want = O.apply_qt(fo, c) if trans == 0 else O.apply_q(fo, c)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(c), trans
    fac.destroy()


def test_residual_and_orthogonality_on_gpu(lib):
    import torch
    m, n, b = 448, 192, 64
    a = _mixed_blr(m, n, b, 7, ((4, 1),), ())
    ref, fac, fo = _factor_both(lib, a, b)
    at = ref.dense()
    e = np.zeros((m, n))
    e[:n] = np.eye(n)
    q1 = lib.to_fortran(torch.from_numpy(e))
    lib.blr_apply_qt(fac, q1, trans=1)
    q1 = q1.cpu().numpy()
    orth = np.linalg.norm(q1.T @ q1 - np.eye(n)) / np.sqrt(n)
    rk, tl = lib.blr_matrix_export(fac)
    r = lib_r_dense(rk, tl, m // b, n // b, b)
    res = np.linalg.norm(q1 @ r - at) / np.linalg.norm(at)
    assert orth <= 1e-12
    assert res <= 1e-13
    # the device R product agrees with the dense R
    x = np.random.default_rng(1).standard_normal((n, 3))
    y = lib.blr_apply_r(fac, lib.to_fortran(torch.from_numpy(x))).cpu().numpy()
    assert np.allclose(y, r @ x, atol=1e-12 * np.abs(r @ x).max())
    fac.destroy()


def test_compression_kernel_parity_fixed_rank(lib):
    """inv1d at 2048 x 1024, b = 128, rank 8 by truncated SVD: tiles equal
    the oracle's best rank-8 approximations."""
    pr = W.inv1d_2048x1024()
    opts = lib.blr_opts_default(b=128, fixed_rank=8, tol=0.0, rec_tol=1e-14)
    mat = lib.blr_compress_kernel(pr.x, pr.y, "inv1d", opts)
    rk, tl = lib.blr_matrix_export(mat)
    p, q, b = 16, 8, 128
    for (i, j) in [(0, 1), (1, 0), (5, 3), (15, 7), (8, 0), (2, 7)]:
        t = lib_tile(rk, tl, p, b, i, j)
        assert t.kind == "L" and t.rank == 8
        want = O.compress_svd(pr.tile(i, j), 8).dense()
        assert np.linalg.norm(t.dense() - want) <= 1e-10 * np.linalg.norm(want), (i, j)
        assert np.allclose(t.u.T @ t.u, np.eye(8), atol=1e-13)
    for i in range(q):
        assert rk[i * p + i] == -1
        assert np.allclose(lib_tile(rk, tl, p, b, i, i).d, pr.tile(i, i), atol=1e-13)
    mat.destroy()


def test_compression_kernel_parity_tolerance(lib):
    """Yukawa 3D at tolerance 1e-8 by truncated pivoted QR: ranks equal the
    oracle's (or differ by one where a pivot tie flips) and every tile meets
    the tolerance; U orthonormal."""
    pr = W.kernel_problem("yukawa3d", 2048, 1024, 128, 31, 32)
    opts = lib.blr_opts_default(b=128, tol=1e-8)
    mat = lib.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts)
    rk, tl = lib.blr_matrix_export(mat)
    p, q, b = 16, 8, 128
    diffs = 0
    for j in range(q):
        for i in range(p):
            t = lib_tile(rk, tl, p, b, i, j)
            a = pr.tile(i, j)
            if i == j:
                assert t.kind == "D"
                continue
            to = O.compress_qrcp(a, 1e-8, b // 2)
            assert np.linalg.norm(t.dense() - a) <= 1e-8 * np.linalg.norm(a) * (1 + 1e-6)
            if t.kind == "L":
                assert np.allclose(t.u.T @ t.u, np.eye(t.rank), atol=1e-13)
            assert abs(t.rank - to.rank) <= 1 or (t.kind == to.kind == "D")
            diffs += t.rank != to.rank
    assert diffs <= 2
    mat.destroy()


def test_inv1d_pipeline_properties(lib):
    """Config-1 shape end to end on the GPU: compression + factorization of
    the ill-conditioned kernel matrix; Res against A~ at 1e-12, Orth at
    1e-12, R^T R = A~^T A~; the oracle on the same A~ gives the same Res."""
    import torch
    pr = W.inv1d_2048x1024()
    opts = lib.blr_opts_default(b=128, fixed_rank=8, tol=0.0, rec_tol=1e-14)
    mat = lib.blr_compress_kernel(pr.x, pr.y, "inv1d", opts)
    rk, tl = lib.blr_matrix_export(mat)
    at = lib_to_oracle(rk, tl, 16, 8, 128).dense()
    fac = lib.blr_qr(mat, opts)
    m, n = 2048, 1024
    e = np.zeros((m, n))
    e[:n] = np.eye(n)
    q1 = lib.to_fortran(torch.from_numpy(e))
    lib.blr_apply_qt(fac, q1, trans=1)
    q1 = q1.cpu().numpy()
    rk2, tl2 = lib.blr_matrix_export(fac)
    r = lib_r_dense(rk2, tl2, 16, 8, 128)
    res = np.linalg.norm(q1 @ r - at) / np.linalg.norm(at)
    orth = np.linalg.norm(q1.T @ q1 - np.eye(n)) / np.sqrt(n)
    assert res <= 1e-12 and orth <= 1e-12
    gram = at.T @ at
    assert np.linalg.norm(r.T @ r - gram) <= 1e-12 * np.linalg.norm(gram)
    fac.destroy()


def test_lstsq_parity(lib):
    import torch
    m, n, b = 256, 128, 32
    a = _mixed_blr(m, n, b, 3)
    ref, fac, fo = _factor_both(lib, a, b)
    bm = W.gaussian_rhs(m, 3, 9)
    x = lib.blr_lstsq(fac, lib.to_fortran(torch.from_numpy(bm))).cpu().numpy()
    xo = O.lstsq(fo, bm)
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)
    fac.destroy()


def test_lstsq_refinement(lib):
    import torch
    m, n, b = 256, 128, 32
    a = _mixed_blr(m, n, b, 4)
    ref = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    ranks, tiles = oracle_to_lib(ref)
    mat = lib.blr_matrix_import(m, n, b, ranks, tiles)
    keep = lib.blr_matrix_clone(mat)
    fac = lib.blr_qr(mat, lib.blr_opts_default(b=b, tol=1e-6, rec_tol=1e-6))
    bm = W.gaussian_rhs(m, 2, 10)
    bt = lib.to_fortran(torch.from_numpy(bm))
    x0 = lib.blr_lstsq(fac, bt).cpu().numpy()
    x1 = lib.blr_lstsq(fac, bt, a_orig=keep, refine_steps=2).cpu().numpy()
    at = ref.dense()
    xs = np.linalg.lstsq(at, bm, rcond=None)[0]
    assert np.linalg.norm(x1 - xs) <= np.linalg.norm(x0 - xs) + 1e-12
    assert np.linalg.norm(x1 - xs) <= 1e-9 * np.linalg.norm(xs)
    fac.destroy()
    keep.destroy()


def test_invalid_arguments_fail_loudly(lib):
    import torch
    a = lib.to_fortran(torch.zeros(64, 128, dtype=torch.float64))
    with pytest.raises(lib.BLRError) as e:
        lib.blr_compress_dense(a, lib.blr_opts_default(b=32, tol=1e-8))
    assert e.value.code == 1          # m < n
    a = lib.to_fortran(torch.zeros(96, 48, dtype=torch.float64))
    with pytest.raises(lib.BLRError):
        lib.blr_compress_dense(a, lib.blr_opts_default(b=40, tol=1e-8))   # b not a multiple of 32
    with pytest.raises(lib.BLRError):
        lib.blr_compress_dense(a, lib.blr_opts_default(b=32, tol=0.0))    # no tolerance, no rank


# ---------------------------------------------------------------- mixed precision
# FP32 trailing updates and recompression, FP64 panels.  Tolerances follow
# from FP32 rounding (u = 6e-8) times the growth of a few hundred updates:
# Orth <= 1e-6 (the mixed-precision target), Res <= 10 x the recompression
# tolerance, R within 1e-5 of the FP64 oracle on well-conditioned inputs.

MIXED_CASES = CASES[:4] + [
    (1024, 512, 256, 6, ((2, 0), (3, 1)), ()),      # b > 128: grouped tensor-core TSQRT updates
]


@pytest.mark.parametrize("m,n,b,seed,dense,zero", MIXED_CASES)
def test_mixed_precision_factor_close_to_oracle(lib, m, n, b, seed, dense, zero):
    import torch
    a = _mixed_blr(m, n, b, seed, dense, zero)
    p, q = m // b, n // b
    ref = O.compress(tiles_of(a, b), p, q, b, eps=1e-14)
    ranks, tiles = oracle_to_lib(ref)
    mat = lib.blr_matrix_import(m, n, b, ranks, tiles)
    opts = lib.blr_opts_default(b=b, tol=1e-6, rec_tol=1e-6, precision=lib.BLR_PREC_MIXED)
    fac = lib.blr_qr(mat, opts)
    fo = O.blr_qr(ref, 1e-14)
    rk, tl = lib.blr_matrix_export(fac)
    r_g = lib_r_dense(rk, tl, p, q, b)
    r_o = fo.r_dense()
    assert np.linalg.norm(r_g - r_o) <= 1e-5 * np.linalg.norm(r_o)
    at = ref.dense()
    e = np.zeros((m, n))
    e[:n] = np.eye(n)
    q1 = lib.to_fortran(torch.from_numpy(e))
    lib.blr_apply_qt(fac, q1, trans=1)
    q1 = q1.cpu().numpy()
    orth = np.linalg.norm(q1.T @ q1 - np.eye(n)) / np.sqrt(n)
    res = np.linalg.norm(q1 @ r_g - at) / np.linalg.norm(at)
    assert orth <= 1e-6
    assert res <= 1e-5
    fac.destroy()


def test_mixed_precision_kernel_matrix(lib):
    """Yukawa 3D, 4096 x 2048, b = 128, tol 1e-6: mixed Res against A within
    10 x tol, Orth <= 1e-6, and the FP64 path on the same input agrees."""
    import torch
    pr = W.kernel_problem("yukawa3d", 4096, 2048, 128, 41, 42)
    out = {}
    for prec in (lib.BLR_PREC_FP64, lib.BLR_PREC_MIXED):
        opts = lib.blr_opts_default(b=128, tol=1e-6, precision=prec)
        mat = lib.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts)
        fac = lib.blr_qr(mat, opts)
        m, n = 4096, 2048
        z = np.random.default_rng(3).standard_normal((n, 8))
        rz = lib.blr_apply_r(fac, lib.to_fortran(torch.from_numpy(z)))
        y = torch.zeros((8, m), dtype=torch.float64, device="cuda").t()
        y[:n] = rz
        lib.blr_apply_qt(fac, y, trans=1)
        az = pr.dense() @ z
        res = np.linalg.norm(y.cpu().numpy() - az) / np.linalg.norm(az)
        e = np.zeros((m, 64))
        e[:64, :64] = np.eye(64)
        e[:n] = np.random.default_rng(4).standard_normal((n, 64))
        qe = lib.to_fortran(torch.from_numpy(e))
        lib.blr_apply_qt(fac, qe, trans=1)
        lib.blr_apply_qt(fac, qe, trans=0)
        orth_probe = np.linalg.norm(qe.cpu().numpy() - e) / np.linalg.norm(e)
        out[prec] = (res, orth_probe)
        fac.destroy()
    assert out[lib.BLR_PREC_FP64][0] <= 1e-5 and out[lib.BLR_PREC_MIXED][0] <= 1e-5
    assert out[lib.BLR_PREC_FP64][1] <= 1e-13 and out[lib.BLR_PREC_MIXED][1] <= 1e-6


def test_strong_admissibility_keeps_near_tiles_dense(lib):
    """Strong admissibility (Section 3.1, eta): a tile whose row and column
    clusters' bounding boxes are closer than eta times the larger diameter
    is stored dense; every other off-diagonal tile is compressed as before
    (dense only when its rank exceeds the threshold).  The factorization of
    the result still meets the tolerance."""
    import torch
    pr = W.kernel_problem("yukawa3d", 2048, 1024, 128, 61, 62)
    p, q, b = 16, 8, 128

    def boxes(pts, nclust):
        return [(pts[:, c * b:(c + 1) * b].min(axis=1), pts[:, c * b:(c + 1) * b].max(axis=1)) for c in range(nclust)]

    bx, by = boxes(pr.x, p), boxes(pr.y, q)
    for eta in (0.5, 2.0):
        opts = lib.blr_opts_default(b=b, tol=1e-8, eta=eta)
        mat = lib.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts)
        rk, tl = lib.blr_matrix_export(mat)
        weak = lib.blr_compress_kernel(pr.x, pr.y, "yukawa3d", lib.blr_opts_default(b=b, tol=1e-8))
        rk0, _ = lib.blr_matrix_export(weak)
        n_forced = 0
        for j in range(q):
            for i in range(p):
                (ilo, ihi), (jlo, jhi) = bx[i], by[j]
                gap = np.maximum(0.0, np.maximum(jlo - ihi, ilo - jhi))
                diam = max(np.linalg.norm(ihi - ilo), np.linalg.norm(jhi - jlo))
                near = np.linalg.norm(gap) < eta * diam
                t = j * p + i
                if i == j or near:
                    assert rk[t] == -1, (eta, i, j)
                    n_forced += i != j
                else:
                    assert rk[t] == rk0[t], (eta, i, j)
        assert n_forced > 0
        fac = lib.blr_qr(mat, opts)
        z = np.random.default_rng(5).standard_normal((1024, 4))
        rz = lib.blr_apply_r(fac, lib.to_fortran(torch.from_numpy(z)))
        y = torch.zeros((4, 2048), dtype=torch.float64, device="cuda").t()
        y[:1024] = rz
        lib.blr_apply_qt(fac, y, trans=1)
        az = pr.dense() @ z
        assert np.linalg.norm(y.cpu().numpy() - az) <= 1e-7 * np.linalg.norm(az)
        fac.destroy()
        weak.destroy()
