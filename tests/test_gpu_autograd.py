"""Differentiable BLR least squares (x = argmin ||A~ x - B||, the least
squares use of A = QR): gradients with respect to B and to the tile
storage (dense blocks, U and V of low-rank tiles) against

* a dense FP64 autograd reference: A~ assembled from the same tiles with
  torch operations (A_ij = U V^T), x by torch's Householder QR and a
  triangular solve, gradients by torch.autograd;
* central finite differences (h = 1e-6) along seeded random directions in
  the space of the live tile entries.  The library's format keeps each U
  orthonormal (the factorization relies on it, Section 3.1); a direction
  that moved U off the orthonormal matrices would change the function the
  factorization computes at first order, so the U part of every direction
  is taken orthogonal to U's columns (then U^T U changes only at O(h^2)).

The loss is L = <W, x> with a seeded W.  Tolerances: the factorization of A~
is run at recompression tolerance 1e-14, so the BLR path is exact up to
rounding amplified by kappa(A~)^2 (z = (A~^T A~)^{-1} xbar); the finite
differences carry O(h^2) truncation and O(u/h) rounding error.
"""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import oracle_to_lib, tiles_of

pytestmark = pytest.mark.gpu


def _tiles_from_dense(a, b, eps):
    m, n = a.shape
    ref = O.compress(tiles_of(a, b), m // b, n // b, b, eps=eps)
    return oracle_to_lib(ref)


def _problem_random(seed):
    m, n, b = 256, 128, 32
    rng = np.random.default_rng(seed)
    a = W.random_blr_dense(m, n, b, 2, seed)
    a[3 * b:4 * b, 1 * b:2 * b] = rng.standard_normal((b, b))       # a dense off-diagonal tile
    ranks, tiles = _tiles_from_dense(a, b, 1e-14)
    return m, n, b, ranks, tiles


def _problem_yukawa():
    # the 4096 x 2048 verification instance: Yukawa kernel, b = 256, tol 1e-8
    pr = W.kernel_problem("yukawa3d", 4096, 2048, 256, 511, 512)
    ranks, tiles = _tiles_from_kernel(pr)
    return 4096, 2048, 256, ranks, tiles


def _tiles_from_kernel(pr):
    from paper_2208_06194_gb300 import blr
    opts = blr.blr_opts_default(b=pr.b, tol=1e-8)
    mat = blr.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts)
    ranks, tiles = blr.blr_matrix_export(mat)
    mat.destroy()
    return ranks, tiles


def _dense_from_tiles(torch, tiles, ranks, m, n, b):
    """A~ from the tile storage with differentiable torch operations."""
    p, q, cap = m // b, n // b, b // 2
    cols = []
    for j in range(q):
        blocks = []
        for i in range(p):
            t = tiles[(j * p + i) * b * b:(j * p + i + 1) * b * b]
            r = int(ranks[j * p + i])
            if r < 0:
                blocks.append(t.reshape(b, b).t())                    # column-major block
            else:
                u = t[:b * r].reshape(r, b).t()
                v = t[b * cap:b * cap + b * r].reshape(r, b).t()
                blocks.append(u @ v.t())
        cols.append(torch.cat(blocks, 0))
    return torch.cat(cols, 1)


def _live_mask(ranks, m, n, b):
    p, q, cap = m // b, n // b, b // 2
    mask = np.zeros(p * q * b * b, dtype=bool)
    for t, r in enumerate(ranks):
        base = t * b * b
        if r < 0:
            mask[base:base + b * b] = True
        else:
            mask[base:base + b * r] = True
            mask[base + b * cap:base + b * cap + b * r] = True
    return mask


def _reference(torch, tiles_np, ranks, bm, wt, m, n, b):
    t = torch.tensor(tiles_np, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch.tensor(bm, dtype=torch.float64, device="cuda", requires_grad=True)
    a = _dense_from_tiles(torch, t, ranks, m, n, b)
    qm, rm = torch.linalg.qr(a)
    x = torch.linalg.solve_triangular(rm, qm.t() @ bt, upper=True)
    loss = (x * wt).sum()
    loss.backward()
    return x.detach(), t.grad.detach(), bt.grad.detach()


def _ours(torch, lib, tiles_np, ranks, bm, m, n, b, refine=2, need_grad=True):
    from paper_2208_06194_gb300.autograd import blr_lstsq_autograd
    t = torch.tensor(tiles_np, dtype=torch.float64, device="cuda", requires_grad=need_grad)
    bt = torch.tensor(bm, dtype=torch.float64, device="cuda", requires_grad=need_grad)
    opts = lib.blr_opts_default(b=b, tol=1e-14, rec_tol=1e-14)
    x = blr_lstsq_autograd(t, bt, ranks, m, n, b, opts, refine)
    return x, t, bt


@pytest.mark.parametrize("which", ["random", "yukawa"])
def test_lstsq_gradients_match_dense_autograd(lib, which):
    import torch
    m, n, b, ranks, tiles = _problem_random(7) if which == "random" else _problem_yukawa()
    nrhs = 3 if which == "random" else 16
    rng = np.random.default_rng(12)
    bm = rng.standard_normal((m, nrhs))
    wt = torch.tensor(rng.standard_normal((n, nrhs)), device="cuda")
    x_ref, g_ref, gb_ref = _reference(torch, tiles, ranks, bm, wt, m, n, b)
    x, t, bt = _ours(torch, lib, tiles, ranks, bm, m, n, b)
    (x * wt).sum().backward()
    tol = 1e-9 if which == "random" else 1e-6
    assert float(torch.linalg.norm(x.detach() - x_ref) / torch.linalg.norm(x_ref)) <= tol
    assert float(torch.linalg.norm(bt.grad - gb_ref) / torch.linalg.norm(gb_ref)) <= tol
    assert float(torch.linalg.norm(t.grad - g_ref) / torch.linalg.norm(g_ref)) <= tol
    mask = torch.tensor(~_live_mask(ranks, m, n, b), device="cuda")
    assert float(t.grad[mask].abs().max()) == 0.0            # nothing outside the live tile entries


def test_lstsq_gradients_match_finite_differences(lib):
    import torch
    m, n, b, ranks, tiles = _problem_random(8)
    nrhs, h = 2, 1e-6
    rng = np.random.default_rng(13)
    bm = rng.standard_normal((m, nrhs))
    wt = torch.tensor(rng.standard_normal((n, nrhs)), device="cuda")
    x, t, bt = _ours(torch, lib, tiles, ranks, bm, m, n, b)
    (x * wt).sum().backward()
    live = _live_mask(ranks, m, n, b)

    def loss(tl, bb):
        xx, _, _ = _ours(torch, lib, tl, ranks, bb, m, n, b, refine=3, need_grad=False)
        return float((xx * wt).sum())

    p, cap = m // b, b // 2
    for k in range(3):
        d = np.where(live, rng.standard_normal(tiles.shape), 0.0)
        for tt, r in enumerate(ranks):
            if r > 0:
                u = tiles[tt * b * b:tt * b * b + b * r].reshape(r, b).T
                g = d[tt * b * b:tt * b * b + b * r].reshape(r, b).T
                d[tt * b * b:tt * b * b + b * r] = (g - u @ (u.T @ g)).T.ravel()
        db = rng.standard_normal(bm.shape)
        fd = (loss(tiles + h * d, bm + h * db) - loss(tiles - h * d, bm - h * db)) / (2 * h)
        an = float((t.grad.cpu().numpy() * d).sum() + (bt.grad.cpu().numpy() * db).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, fd, an)


def test_solve_r_both_directions(lib):
    import torch
    m, n, b, ranks, tiles = _problem_random(9)
    fac = lib.blr_qr(lib.blr_matrix_import(m, n, b, ranks, tiles), lib.blr_opts_default(b=b, tol=1e-14))
    rk, tl = lib.blr_matrix_export(fac)
    from tests.helpers import lib_r_dense
    r = lib_r_dense(rk, tl, m // b, n // b, b)
    c = np.random.default_rng(3).standard_normal((n, 4))
    x0 = lib.blr_solve_r(fac, lib.to_fortran(torch.from_numpy(c)), trans=0).cpu().numpy()
    x1 = lib.blr_solve_r(fac, lib.to_fortran(torch.from_numpy(c)), trans=1).cpu().numpy()
    assert np.linalg.norm(r @ x0 - c) <= 1e-11 * np.linalg.norm(c)
    assert np.linalg.norm(r.T @ x1 - c) <= 1e-11 * np.linalg.norm(c)
    fac.destroy()
