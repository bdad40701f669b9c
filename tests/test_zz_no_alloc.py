"""blr_apply_qt_noalloc: the allocation-free variant of blr_apply_qt for
callers that cannot allocate device memory during a call (applications that
own all device memory through their own pool, latency-critical solvers that
cannot afford the allocator's implicit synchronisation).  It must give the
allocating call's result, on consecutive calls that reuse its static
scratch, accept right-hand-side counts up to what that scratch holds and
reject one column group more.  Collected last so that a failure here does
not stop the other tests."""
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
    # the exact limit of the documented formula: 256 bytes + q*8 rounded up
    # to 256 + ceil(nrhs/8) * (16 (b/2) + 64) * 8 bytes <= 4 MiB
    q = n // b
    fixed = 256 + (q * 8 + 255) // 256 * 256
    per_group = (16 * (b // 2) + 64) * 8
    groups = (4 * 2 ** 20 - fixed) // per_group
    nmax = groups * 8
    c = rng.standard_normal((m, nmax))
    want = lib.to_fortran(torch.from_numpy(c))
    lib.blr_apply_qt(fac, want, trans=0)
    got = lib.to_fortran(torch.from_numpy(c))
    lib.blr_apply_qt_noalloc(fac, got, trans=0)                 # the largest accepted count works
    assert float(torch.linalg.norm(got - want) / torch.linalg.norm(want)) <= 1e-13
    over = lib.fortran_empty(m, nmax + 1)                       # one more column group
    with pytest.raises(lib.BLRError) as e:
        lib.blr_apply_qt_noalloc(fac, over, trans=0)
    assert e.value.code == 1
    fac.destroy()
