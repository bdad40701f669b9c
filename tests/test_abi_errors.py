"""Error behaviour of the C ABI, on the host (no GPU needed).

include/blr.h promises that pointers, sizes and options are checked on the
host before any CUDA call (BLR_ERR_INVALID with a message on any machine),
that messages are per thread, and that nothing falls back to the CPU: with
valid arguments and no usable device a call fails with BLR_ERR_CUDA.  The
shape rules are those of Eq. 1 (A = QR with m >= n) and of the p x q tiling
with square b x b tiles (Section 2).

Invalid-argument cases pass NULL, or a pointer that the call rejects before
it could use it.  The no-device cases pass valid arguments, so they run only
where no CUDA device is visible.
"""
import ctypes
import os
import threading

import numpy as np
import pytest

from paper_2208_06194_gb300 import blr

INVALID, CUDA = 1, 3
_P = ctypes.c_void_p


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(blr.LIB_PATH):
        from paper_2208_06194_gb300 import build
        build.build()
    return blr.lib()


def _no_device():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


no_device = pytest.mark.skipif(not _no_device(), reason="a CUDA device is visible")


def _opts(**kw):
    return blr.blr_opts_default(**kw)


def _points(n, dim, seed=0):
    return np.ascontiguousarray(np.random.default_rng(seed).random((n, dim)))


def _compress_kernel(L, x, y, dim, m, n, kid, o):
    out = _P()
    dp = ctypes.POINTER(ctypes.c_double)
    xp = x.ctypes.data_as(dp) if x is not None else None
    yp = y.ctypes.data_as(dp) if y is not None else None
    rc = L.blr_compress_kernel(xp, yp, dim, m, n, kid, None, ctypes.byref(o) if o is not None else None,
                               ctypes.byref(out), None)
    return rc, out


@pytest.mark.parametrize("case,m,n,kid,dim,kw,msg", [
    ("m < n", 128, 256, 1, 3, {"b": 128}, "m >= n"),
    ("m not a multiple of b", 200, 128, 1, 3, {"b": 128}, "multiples of b"),
    ("n = 0", 128, 0, 1, 3, {"b": 128}, "multiples of b"),
    ("b not a multiple of 32", 96 * 4, 96 * 2, 1, 3, {"b": 96 + 8}, "multiple of 32"),
    ("b above the maximum", 8192, 4096, 1, 3, {"b": 4096}, "multiple of 32"),
    ("b = 1024 (tiles above 512 not supported)", 2048, 1024, 1, 3, {"b": 1024}, "[32, 512]"),
    ("unknown kernel", 256, 128, 3, 3, {"b": 128}, "unknown kernel"),
    ("1D kernel with 3D points", 256, 128, 0, 3, {"b": 128}, "dim=1"),
    ("fixed rank above b/2", 256, 128, 1, 3, {"b": 128, "fixed_rank": 65}, "fixed_rank"),
    ("neither rank nor tolerance", 256, 128, 1, 3, {"b": 128, "tol": 0.0}, "tol > 0"),
    ("negative tolerance", 256, 128, 1, 3, {"b": 128, "tol": -1e-8}, "negative"),
    ("negative eta", 256, 128, 1, 3, {"b": 128, "eta": -1.0}, "negative"),
    ("unknown precision", 256, 128, 1, 3, {"b": 128, "precision": 7}, "precision"),
])
def test_compress_kernel_rejects_on_host(L, case, m, n, kid, dim, kw, msg):
    x, y = _points(max(m, 1), dim), _points(max(n, 1), dim, 1)
    rc, out = _compress_kernel(L, x, y, dim, m, n, kid, _opts(**kw))
    assert rc == INVALID, case
    assert out.value is None
    assert msg in blr.blr_last_error(), (case, blr.blr_last_error())


def test_compress_kernel_null_arguments(L):
    x = _points(256, 3)
    assert _compress_kernel(L, None, x, 3, 256, 128, 1, _opts(b=128))[0] == INVALID
    assert _compress_kernel(L, x, None, 3, 256, 128, 1, _opts(b=128))[0] == INVALID
    assert _compress_kernel(L, x, x, 3, 256, 128, 1, None)[0] == INVALID
    assert "NULL" in blr.blr_last_error() or "opts" in blr.blr_last_error()


def test_compress_dense_rejects_on_host(L):
    out = _P()
    o = _opts(b=128)
    assert L.blr_compress_dense(None, 256, 256, 128, ctypes.byref(o), ctypes.byref(out), None) == INVALID
    # a short leading dimension is caught before the (never dereferenced) pointer is used
    fake = _P(0x1000)
    assert L.blr_compress_dense(fake, 255, 256, 128, ctypes.byref(o), ctypes.byref(out), None) == INVALID
    assert "lda" in blr.blr_last_error()
    assert L.blr_compress_dense(fake, 256, 128, 256, ctypes.byref(o), ctypes.byref(out), None) == INVALID
    assert out.value is None


def _import(L, m, n, b, ranks, tiles):
    out = _P()
    rp = ranks.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if ranks is not None else None
    tp = tiles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if tiles is not None else None
    return L.blr_matrix_import(m, n, b, rp, tp, ctypes.byref(out), None), out


@pytest.mark.parametrize("bad_rank", [-2, 17, 1 << 20])
def test_import_rejects_ranks_outside_the_tile_capacity(L, bad_rank):
    b, p, q = 32, 3, 2
    ranks = np.zeros(p * q, dtype=np.int32)
    ranks[4] = bad_rank
    tiles = np.zeros(p * q * b * b)
    rc, out = _import(L, p * b, q * b, b, ranks, tiles)
    assert rc == INVALID and out.value is None
    assert "tile 4" in blr.blr_last_error()


def test_import_rejects_shapes_and_nulls(L):
    ranks = np.zeros(6, dtype=np.int32)
    tiles = np.zeros(6 * 32 * 32)
    assert _import(L, 64, 96, 32, ranks, tiles)[0] == INVALID          # m < n
    assert _import(L, 96, 64, 48, ranks, tiles)[0] == INVALID          # b not a multiple of 32
    assert _import(L, 96, 64, 32, None, tiles)[0] == INVALID
    assert _import(L, 96, 64, 32, ranks, None)[0] == INVALID


def test_qr_entry_points_reject_on_host(L):
    f = _P()
    o = _opts(b=128)
    assert L.blr_qr(None, ctypes.byref(o), ctypes.byref(f), None) == INVALID
    arr = (_P * 2)()
    fs = (_P * 2)()
    assert L.blr_qr_batched(arr, 0, ctypes.byref(o), fs, None) == INVALID
    assert L.blr_qr_batched(None, 2, ctypes.byref(o), fs, None) == INVALID
    plan = _P()
    assert L.blr_batch_plan_create(arr, 2, ctypes.byref(o), ctypes.byref(plan), None) == INVALID
    assert "matrix 0 is NULL" in blr.blr_last_error()
    assert plan.value is None
    bad = _opts(b=128, precision=9)
    assert L.blr_batch_plan_create(arr, 2, ctypes.byref(bad), ctypes.byref(plan), None) == INVALID
    assert "precision" in blr.blr_last_error()
    nortol = _opts(b=128, tol=0.0, rec_tol=0.0)
    assert L.blr_batch_plan_create(arr, 2, ctypes.byref(nortol), ctypes.byref(plan), None) == INVALID
    assert "rec_tol" in blr.blr_last_error()
    for kw, msg in [({"trace": -1}, "trace"), ({"test_withhold": -3}, "test_withhold"),
                    ({"prep_slots": -1}, "prep_slots")]:
        neg = _opts(b=128, **kw)
        assert L.blr_batch_plan_create(arr, 2, ctypes.byref(neg), ctypes.byref(plan), None) == INVALID
        assert msg in blr.blr_last_error()
    assert L.blr_batch_plan_launch(None, None) == INVALID
    assert L.blr_batch_plan_finish(None, None) == INVALID
    assert L.blr_batch_plan_factor(None, 0) is None
    L.blr_batch_plan_destroy(None)
    L.blr_destroy_matrix(None)
    L.blr_destroy_factor(None)


def test_solve_entry_points_reject_null_handles(L):
    fake = _P(0x1000)    # never dereferenced: every call below fails on its NULL handle first
    assert L.blr_apply_qt(None, fake, 128, 1, 0, None) == INVALID
    assert L.blr_apply_qt_noalloc(None, fake, 128, 1, 0, None) == INVALID
    assert L.blr_lstsq(None, None, fake, 128, fake, 128, 1, 0, None) == INVALID
    assert L.blr_matmul(None, fake, 128, fake, 128, 1, None) == INVALID
    assert L.blr_apply_r(None, fake, 128, fake, 128, 1, None) == INVALID
    assert L.blr_solve_r(None, fake, 128, fake, 128, 1, 0, None) == INVALID
    assert L.blr_lstsq_backward(None, None, fake, 128, fake, 128, fake, 128, 1, fake, 128, fake, None) == INVALID
    buf = np.zeros(4)
    assert L.blr_factor_export_t(None, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None) == INVALID
    assert L.blr_matrix_export(None, 0, None, None, None) == INVALID
    st = blr.Stats()
    assert L.blr_stats(None, 0, ctypes.byref(st)) == INVALID
    clone = _P()
    assert L.blr_matrix_clone(None, ctypes.byref(clone), None) == INVALID
    # blr_densify: NULL handle or output, which out of range, R / Y~ of a matrix
    assert L.blr_densify(None, 0, 0, fake, 128, None) == INVALID
    assert L.blr_densify(fake, 0, 0, None, 128, None) == INVALID
    assert L.blr_densify(fake, 1, 3, fake, 128, None) == INVALID
    assert L.blr_densify(fake, 0, 1, fake, 128, None) == INVALID
    assert "matrix handle" in blr.blr_last_error()
    # blr_trace_export: NULL factor, or no buffer for a positive capacity
    assert L.blr_trace_export(None, None, 0, None) == -1
    assert L.blr_trace_export(fake, None, 4, None) == -1


def test_tc_update_bench_rejects_on_host(L):
    ms = ctypes.c_double()
    assert L.blr_tc_update_bench(96, 1, 1, 0, ctypes.byref(ms), None) == INVALID     # b not a multiple of 128
    assert L.blr_tc_update_bench(512, 0, 1, 0, ctypes.byref(ms), None) == INVALID    # no CTA
    assert L.blr_tc_update_bench(512, 1, 1, 5, ctypes.byref(ms), None) == INVALID    # variant not built
    assert L.blr_tc_update_bench(512, 1, 1, 0, None, None) == INVALID


def test_tc_selftest_rejects_on_host(L):
    fake = _P(0x1000)
    assert L.blr_tc_gemm_selftest(None, 128, fake, 8, fake, 128, 128, 8, 8, None) == INVALID
    assert L.blr_tc_gemm_selftest(fake, 127, fake, 8, fake, 128, 128, 8, 8, None) == INVALID   # lda < m
    assert L.blr_tc_gemm_selftest(fake, 128, fake, 7, fake, 128, 128, 8, 8, None) == INVALID   # ldb < k
    assert L.blr_tc_gemm_selftest(fake, 128, fake, 8, fake, 128, 0, 8, 8, None) == INVALID     # m = 0


def test_error_messages_are_per_thread(L):
    seen = {}

    def worker():
        _import(L, 64, 96, 32, np.zeros(6, dtype=np.int32), np.zeros(6 * 1024))
        seen["worker"] = blr.blr_last_error()

    _compress_kernel(L, _points(256, 3), _points(128, 3), 3, 256, 128, 5, _opts(b=128))
    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "m >= n" in seen["worker"]
    assert "unknown kernel" in blr.blr_last_error()


@no_device
def test_valid_compress_without_a_device_fails_loudly(L):
    rc, out = _compress_kernel(L, _points(256, 3), _points(128, 3), 3, 256, 128, 1, _opts(b=128, tol=1e-8))
    assert rc == CUDA and out.value is None
    assert "no usable CUDA device" in blr.blr_last_error()


@no_device
def test_valid_import_without_a_device_fails_loudly(L):
    rc, out = _import(L, 96, 64, 32, np.full(6, -1, dtype=np.int32), np.zeros(6 * 1024))
    assert rc == CUDA and out.value is None
    assert "no usable CUDA device" in blr.blr_last_error()


@no_device
def test_python_binding_raises_without_a_device(L):
    with pytest.raises(blr.BLRError) as e:
        blr.blr_compress_kernel(_points(256, 3).T, _points(128, 3).T, "yukawa3d", _opts(b=128, tol=1e-8),
                                stream=0)
    assert e.value.code == CUDA


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every binding call raises."""
    monkeypatch.setattr(blr, "_lib", None)
    monkeypatch.setattr(blr, "LIB_PATH", str(tmp_path / "libblrqr.so"))
    with pytest.raises(RuntimeError, match="is missing"):
        blr.blr_opts_default()
    with pytest.raises(RuntimeError, match="is missing"):
        blr.blr_dag_selfcheck(2, 1)
