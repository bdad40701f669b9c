"""Batched factorization: several independent BLR matrices of different
shapes and tile sizes in one persistent launch (blr_qr_batched), and the
capturable launch plan replayed from a CUDA graph.  The result of each
matrix must be bit-for-bit the result of its own blr_qr: a tile's writers
run in the order its own DAG fixes, whichever matrices share the launch."""
import numpy as np
import pytest

from oracle import blr_qr as O
from paper_2208_06194_gb300 import workloads as W
from tests.helpers import oracle_to_lib, tiles_of

pytestmark = pytest.mark.gpu

SHAPES = [(256, 128, 32, 1), (448, 192, 64, 2), (384, 384, 128, 3), (640, 256, 128, 4)]


def _mats(lib):
    out = []
    for m, n, b, seed in SHAPES:
        rng = np.random.default_rng(seed)
        a = W.random_blr_dense(m, n, b, 2, seed)
        a[2 * b:3 * b, 0:b] = rng.standard_normal((b, b))        # a dense off-diagonal tile
        ref = O.compress(tiles_of(a, b), m // b, n // b, b, eps=1e-14)
        out.append(oracle_to_lib(ref) + (m, n, b))
    return out


def _import(lib, spec):
    ranks, tiles, m, n, b = spec
    return lib.blr_matrix_import(m, n, b, ranks, tiles)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_launch_equals_separate_launches(lib, prec):
    specs = _mats(lib)
    opts = lib.blr_opts_default(b=512, tol=1e-14, rec_tol=1e-14,
                                precision=lib.BLR_PREC_MIXED if prec == "mixed" else lib.BLR_PREC_FP64)
    single = [lib.blr_qr(_import(lib, s), opts) for s in specs]
    batch = lib.blr_qr_batched([_import(lib, s) for s in specs], opts)
    for f1, f2 in zip(single, batch):
        r1, t1 = lib.blr_matrix_export(f1)
        r2, t2 = lib.blr_matrix_export(f2)
        assert np.array_equal(r1, r2)
        assert np.array_equal(t1, t2)
        assert np.array_equal(lib.blr_factor_export_t(f1), lib.blr_factor_export_t(f2))
    st = lib.blr_stats(batch[0])
    assert st["tasks"][0] == sum(n // b for _, n, b, _ in SHAPES)      # every matrix's GEQRTs ran
    for f in single + batch:
        f.destroy()


def test_plan_replayed_from_a_cuda_graph(lib):
    import torch
    specs = _mats(lib)
    opts = lib.blr_opts_default(b=512, tol=1e-14, rec_tol=1e-14, precision=lib.BLR_PREC_MIXED)
    want = [lib.blr_matrix_export(lib.blr_qr(_import(lib, s), opts)) for s in specs]
    inputs = [_import(lib, s) for s in specs]
    plan = lib.BatchPlan(inputs, opts)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan.launch(stream=side.cuda_stream)      # first launch outside the capture
        plan.finish(stream=side.cuda_stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        plan.launch(stream=side.cuda_stream)
    for _ in range(2):                            # replays re-factor the same inputs
        graph.replay()
        plan.finish(stream=side.cuda_stream)
        for i, (r0, t0) in enumerate(want):
            r, t = lib.blr_matrix_export(plan.factor(i))
            assert np.array_equal(r, r0) and np.array_equal(t, t0), i
    # the inputs were not consumed
    r_in, t_in = lib.blr_matrix_export(inputs[0])
    assert np.array_equal(r_in, specs[0][0]) and np.array_equal(t_in, specs[0][1])
    del graph
    plan.destroy()
    for m in inputs:
        m.destroy()
