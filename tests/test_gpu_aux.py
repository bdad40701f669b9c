"""Auxiliary subsystems on the GPU: the scheduler watchdog (a device wait
that runs out and returns BLR_ERR_TIMEOUT, with the context still usable),
the per-task trace, and densification of BLR storage."""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import lib_r_dense, lib_to_oracle, lib_y_dense, oracle_to_lib, tiles_of

pytestmark = pytest.mark.gpu


def _small(lib, seed=31, m=256, n=128, b=32):
    a = W.random_blr_dense(m, n, b, 2, seed)
    ref = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    ranks, tiles = oracle_to_lib(ref)
    return ref, lambda: lib.blr_matrix_import(m, n, b, ranks, tiles)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("withheld", ["geqrt0", "tpmqrt"])
def test_watchdog_ends_a_stalled_scheduler(lib, prec, withheld):
    """One task of a tiny DAG releases none of its successors (the test
    hook): the remaining tasks never become ready, every scheduler CTA waits
    on an empty queue until the 100 ms watchdog runs out, and blr_qr returns
    BLR_ERR_TIMEOUT.  The next factorization in the same process succeeds
    and matches the oracle."""
    import time
    import torch
    ref, make = _small(lib)
    p, q = 8, 4
    if withheld == "geqrt0":
        task = 0
    else:
        task = next(t for t in range(10 ** 6) if lib.blr_dag_task(p, q, t)[0] == (3, 2, 1, 0))
    precision = lib.BLR_PREC_MIXED if prec == "mixed" else lib.BLR_PREC_FP64
    opts = lib.blr_opts_default(b=32, tol=1e-14, rec_tol=1e-14, precision=precision, watchdog_ms=100,
                                test_withhold=task + 1)
    t0 = time.time()
    with pytest.raises(lib.BLRError) as e:
        lib.blr_qr(make(), opts)
    assert e.value.code == 4, str(e.value)
    assert "watchdog" in str(e.value)
    assert time.time() - t0 < 30.0
    torch.cuda.synchronize()
    opts.test_withhold = 0
    opts.watchdog_ms = 0
    fac = lib.blr_qr(make(), opts)
    rk, tl = lib.blr_matrix_export(fac)
    r_g = lib_r_dense(rk, tl, p, q, 32)
    r_o = O.blr_qr(ref, 1e-14).r_dense()
    tol = 1e-5 if prec == "mixed" else 1e-11
    assert np.linalg.norm(r_g - r_o) <= tol * np.linalg.norm(r_o)
    fac.destroy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_trace_records_every_task_in_dependency_order(lib, prec):
    """opts.trace: one event per task, the task set equals the DAG's, and no
    task starts before a predecessor ended (an update QR releases the next
    one of its column after its first 128-column group, so that edge is
    exempt; the next one starts after it did)."""
    ref, make = _small(lib, seed=33)
    p, q = 8, 4
    precision = lib.BLR_PREC_MIXED if prec == "mixed" else lib.BLR_PREC_FP64
    opts = lib.blr_opts_default(b=32, tol=1e-14, rec_tol=1e-14, precision=precision, trace=100000)
    fac = lib.blr_qr(make(), opts)
    events, total = lib.blr_trace_export(fac)
    n_tasks = q + sum(q - k - 1 for k in range(q)) + sum(p - k - 1 for k in range(q)) + \
        sum((p - k - 1) * (q - k - 1) for k in range(q))
    assert total == n_tasks and len(events) == n_tasks
    want = {lib.blr_dag_task(p, q, t)[0]: t for t in range(n_tasks)}
    got = {(e["type"], e["i"], e["j"], e["k"]): e for e in events}
    assert set(got) == set(want)
    for key, t in want.items():
        e = got[key]
        assert e["t_end_ns"] >= e["t_start_ns"] and 0 <= e["cta"] and e["matrix"] == 0
        for sid in lib.blr_dag_task(p, q, t)[1]:
            s = got[lib.blr_dag_task(p, q, sid)[0]]
            if key[0] == 2 and s["type"] == 2:
                assert s["t_start_ns"] >= e["t_start_ns"], (key, s)
                continue
            assert s["t_start_ns"] >= e["t_end_ns"], (key, s)
    ct = lib.chrome_trace(events)
    assert len(ct["traceEvents"]) == n_tasks and all(ev["dur"] >= 0 for ev in ct["traceEvents"])
    # a smaller capacity keeps the first events and still counts every task
    opts.trace = 10
    fac2 = lib.blr_qr(make(), opts)
    ev2, total2 = lib.blr_trace_export(fac2)
    assert len(ev2) == 10 and total2 == n_tasks
    fac.destroy()
    fac2.destroy()


def test_densify_matrix_r_and_reflectors(lib):
    """blr_densify of a matrix (A~), and of a factor's R and Y~, against the
    same storage densified on the host."""
    m, n, b = 448, 192, 64
    p, q = m // b, n // b
    a = W.random_blr_dense(m, n, b, 3, seed=35)
    a[4 * b:5 * b, b:2 * b] = np.random.default_rng(36).standard_normal((b, b))   # a dense off-diagonal tile
    ref = O.compress(tiles_of(a, b), p, q, b, eps=1e-14)
    ranks, tiles = oracle_to_lib(ref)
    mat = lib.blr_matrix_import(m, n, b, ranks, tiles)
    d = lib.blr_densify(mat, 0).cpu().numpy()
    want = ref.dense()
    assert np.allclose(d, want, rtol=0, atol=1e-13 * np.abs(want).max())
    fac = lib.blr_qr(mat, lib.blr_opts_default(b=b, tol=1e-14, rec_tol=1e-14))
    rk, tl = lib.blr_matrix_export(fac)
    r = lib.blr_densify(fac, 1).cpu().numpy()
    r_h = lib_r_dense(rk, tl, p, q, b)
    assert r.shape == (n, n) and np.allclose(r, r_h, rtol=0, atol=1e-13 * np.abs(r_h).max())
    assert np.array_equal(np.tril(r, -1), np.zeros_like(r))
    y = lib.blr_densify(fac, 2).cpu().numpy()
    for k in range(q):
        for i in range(p):
            blk = y[i * b:(i + 1) * b, k * b:(k + 1) * b]
            if i < k:
                assert not blk.any()
            else:
                yh = lib_y_dense(rk, tl, p, b, i, k)
                assert np.allclose(blk, yh, rtol=0, atol=1e-13 * max(1.0, np.abs(yh).max())), (i, k)
    st = lib.blr_densify(fac, 0).cpu().numpy()
    assert np.allclose(st, lib_to_oracle(rk, tl, p, q, b).dense(), rtol=0, atol=1e-13 * np.abs(st).max())
    fac.destroy()
