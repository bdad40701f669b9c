"""The 65536 x 32768 Yukawa workload at full size, in the launch
configuration bench.py times (mixed precision, tol 1e-5, dense threshold 16),
and the FP64 path at 16384 x 8192: properties that hold at any size, plus
sampled outputs the oracle computes one by one.

* Res_A = ||Q R - A||_F / ||A||_F <= 10 tol and Orth = ||Q^T Q - I||_F/sqrt(n)
  (<= 1e-6 mixed, <= 1e-12 FP64), estimated with Gaussian probes
  (E||M Z||^2 = k ||M||^2) against the uncompressed kernel matrix;
* compression of sampled tiles against the oracle's truncated pivoted QR of
  the same tile (ranks equal up to a pivot tie, so a tile whose rank is at
  the dense threshold may land on either side of it; error within tol, U
  orthonormal);
* R_kk upper triangular with a finite nonzero diagonal for sampled k.
"""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import lib_tile

pytestmark = pytest.mark.gpu


def _probe(lib, pr, opts, k=8):
    import torch
    import bench
    mat = lib.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts)
    keep = lib.blr_matrix_clone(mat)
    fac = lib.blr_qr(mat, opts)
    res_a, res_at, orth = bench.probes(lib, fac, keep, pr, torch, torch.device("cuda", 0), k=k)
    return keep, fac, res_a, orth


def test_full_size_mixed_in_bench_configuration(lib):
    tol, dense = 1e-5, 16
    pr = W.yukawa3d(65536, 32768, 512, 301, 302)
    opts = lib.blr_opts_default(b=512, tol=tol, precision=lib.BLR_PREC_MIXED, dense_rank=dense)
    keep, fac, res_a, orth = _probe(lib, pr, opts)
    assert res_a <= 10 * tol, res_a
    assert orth <= 1e-6, orth
    rk, tl = lib.blr_matrix_export(keep)
    p, b = 128, 512
    for (i, j) in [(1, 0), (77, 5), (127, 63), (40, 20), (3, 60)]:
        t = lib_tile(rk, tl, p, b, i, j)
        a = pr.tile(i, j)
        ref = O.compress_qrcp(a, tol, b // 2)          # the oracle's rank, no threshold
        r_ref = ref.rank if ref.kind == "L" else b // 2 + 1
        assert np.linalg.norm(t.dense() - a) <= tol * np.linalg.norm(a) * (1 + 1e-6), (i, j)
        if t.kind == "L":
            assert t.rank <= dense and abs(t.rank - r_ref) <= 1, (i, j, t.rank, r_ref)
            assert np.allclose(t.u.T @ t.u, np.eye(t.rank), atol=1e-12)
        else:
            assert r_ref >= dense, (i, j, r_ref)     # dense: the rank is at or above the threshold
    rf, tf = lib.blr_matrix_export(fac)
    for k in (0, 31, 63):
        r = lib_tile(rf, tf, p, b, k, k).d
        d = np.diag(r)
        assert np.all(np.isfinite(d)) and np.all(d != 0.0)
    fac.destroy()
    keep.destroy()


def test_fp64_path_at_16384x8192(lib):
    tol = 1e-6
    pr = W.yukawa3d(16384, 8192, 512, 301, 302)
    opts = lib.blr_opts_default(b=512, tol=tol, precision=lib.BLR_PREC_FP64, dense_rank=128)
    keep, fac, res_a, orth = _probe(lib, pr, opts)
    assert res_a <= 10 * tol, res_a
    assert orth <= 1e-12, orth
    fac.destroy()
    keep.destroy()
