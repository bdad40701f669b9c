"""blr_apply_qt_noalloc: the allocation-free variant of blr_apply_qt for
callers that cannot allocate device memory during a call (allocation-free
stream captures, application-owned memory pools, latency-critical solvers).
It must give the allocating call's result, on consecutive calls that reuse
its static scratch, and reject right-hand-side counts beyond that scratch.
Collected last so that a failure here does not stop the other tests."""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import oracle_to_lib, tiles_of

pytestmark = pytest.mark.gpu


def test_apply_qt_noalloc_matches_allocating_call(lib):
    import torch
    m, n, b = 448, 192, 64
    a = W.random_blr_dense(m, n, b, 2, seed=21)
    ref = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
    ranks, tiles = oracle_to_lib(ref)
    fac = lib.blr_qr(lib.blr_matrix_import(m, n, b, ranks, tiles),
                     lib.blr_opts_default(b=b, tol=1e-14, rec_tol=1e-14))
    rng = np.random.default_rng(22)
    for call, (trans, nrhs) in enumerate([(0, 13), (1, 5)]):
        c = rng.standard_normal((m, nrhs))
        want = lib.to_fortran(torch.from_numpy(c))
        lib.blr_apply_qt(fac, want, trans=trans)
        got = lib.to_fortran(torch.from_numpy(c))
        lib.blr_apply_qt_noalloc(fac, got, trans=trans)
        err = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
        assert err <= 1e-13, (call, err)
    big = lib.fortran_empty(m, 8192)   # 1024 column groups x 4.6 KB > 4 MiB at b = 64
    with pytest.raises(lib.BLRError) as e:
        lib.blr_apply_qt_noalloc(fac, big, trans=0)
    assert e.value.code == 1
    fac.destroy()
