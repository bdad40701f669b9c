"""The tcgen05 tensor-core building block of the mixed-precision updates,
checked in isolation: D = A B with 3xTF32 products (x = hi + lo, both TF32)
and FP32 accumulation in TMEM.  The elementwise bound is what that
arithmetic guarantees: the dropped lo*lo term and the TF32 rounding of lo
(each 2^-22 relative to |a||b|) plus FP32 accumulation over K terms; it is
about 2^11 times tighter than a single TF32 product, so it also shows that
the lo parts are used."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,seed", [
    (128, 256, 32, 1),      # one tile, one K chunk
    (128, 16, 8, 2),        # smallest N, partial K chunk
    (300, 200, 77, 3),      # ragged M, N (not a multiple of 16) and K
    (512, 512, 512, 4),     # several tiles in both directions, 16 K chunks
])
def test_tc_gemm_matches_fp64(lib, m, n, k, seed):
    import torch
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((k, n))
    d = lib.blr_tc_gemm_selftest(lib.to_fortran(torch.from_numpy(a)), lib.to_fortran(torch.from_numpy(b)))
    got = d.cpu().numpy()
    want = a @ b
    scale = np.abs(a) @ np.abs(b)
    bound = (2.0 ** -20 + k * 2.0 ** -23) * scale
    assert np.all(np.abs(got - want) <= bound), float(np.max(np.abs(got - want) / scale))


def test_tc_gemm_rejects_bad_shapes(lib):
    import torch
    a = lib.fortran_empty(64, 32)
    b = lib.fortran_empty(16, 8)       # inner dimensions differ
    with pytest.raises(ValueError):
        lib.blr_tc_gemm_selftest(a, b)


def test_dense_update_bench_runs_every_variant(lib):
    """The diagnostic timing of the dense prepared update runs each built
    variant to completion (a tensor-core wait that ran out would raise)."""
    for v in (0, 1, 2, 3, 4, 6, 9, 11, 15, 17, 19):
        r = lib.blr_tc_update_bench(b=256, ctas=4, reps=2, variant=v)
        assert r["ms_per_update"] > 0 and r["aggregate_tflops"] > 0
