"""Host-side checks that need no GPU: the library loads and exports every
entry point declared in include/blr.h, and the scheduler's DAG formulas
(shared by host and device code) pass the host self-check."""
import os
import re

import pytest

from paper_2208_06194_gb300 import blr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "blr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blr_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(blr.LIB_PATH):
        from paper_2208_06194_gb300 import build
        build.build()
    return blr.lib()


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert "blr_qr" in names and "blr_compress_kernel" in names and "blr_lstsq" in names
    for name in names:
        assert hasattr(built, name), name
    for name in names:
        assert name in blr.EXPORTED, f"binding lacks {name}"


def test_opts_default_is_host_only(built):
    o = blr.blr_opts_default()
    assert o.b == 512 and o.tol == 1e-8 and o.precision == blr.BLR_PREC_FP64


@pytest.mark.parametrize("p,q", [(1, 1), (2, 1), (3, 3), (5, 2), (16, 8), (17, 9), (64, 32)])
def test_dag_formulas_host_selfcheck(built, p, q):
    for seed in range(4):
        assert blr.blr_dag_selfcheck(p, q, seed) == 0


def test_dag_selfcheck_rejects_bad_shape(built):
    assert blr.blr_dag_selfcheck(2, 3, 0) != 0


@pytest.mark.parametrize("shapes", [[(1, 1)], [(3, 2), (8, 4)], [(16, 8), (5, 5), (2, 1), (64, 32)],
                                    [(12, 6)] * 7])
def test_batch_task_numbering_host_selfcheck(built, shapes):
    ps, qs = zip(*shapes)
    for seed in range(3):
        assert blr.blr_batch_selfcheck(ps, qs, seed) == 0


def test_batch_selfcheck_rejects_bad_shapes(built):
    assert blr.blr_batch_selfcheck([2, 3], [1, 4], 0) != 0
