"""Planted mistakes in the oracle, on the CPU: each pin must catch them.

A mutant is one oracle (or input-generator) function recompiled from its
own source with one plausible slip (a dropped term, a wrong sign, a
transposed operand, an off-by-one, a wrong loop order) and patched into the
modules that bind it for the duration of one test.  The pins of tests/test_oracle.py named beside it must
then fail; without a mutant they pass (that file's own run).
"""
import inspect
import textwrap

import pytest

from oracle import blr_qr as O
from oracle import dense_qr as D
from paper_2208_06194_gb300 import workloads as W
from tests import test_oracle as T


def _fails(fn, *args):
    try:
        fn(*args)
    except Exception:
        return True
    return False


def _tpmqrt_all_kinds():
    for y in "LD":
        for r in "LD":
            for a in "LD":
                T.test_tpmqrt_equals_dense_trapezoidal_reflector(y, r, a)


def _tsqrt_all_tails():
    for rows in (0, 1, 3, 8):
        T.test_tsqrt_update_qr(rows)


def _reflector_cases():
    for x in ([3.0, 4.0], [-3.0, 4.0, 0.0], [0.0, 1.0, 2.0], [2.0, 0.0, 0.0]):
        T.test_reflector_maps_to_beta_e1(x)


PINS = {
    "reflector": _reflector_cases,
    "lapack": T.test_dense_qr_matches_lapack,
    "geqrt_wy": T.test_geqrt_compact_wy_equals_product_of_reflectors,
    "tsqrt": _tsqrt_all_tails,
    "larfb": T.test_larfb_is_qt_times_c,
    "tpmqrt": _tpmqrt_all_kinds,
    "truncation_rank": T.test_truncation_rank_closed_form,
    "rounded_addition": T.test_rounded_addition_bound_orthonormal_and_rank,
    "op3_op4": T.test_op3_op4_products,
    "compress": T.test_compress_qrcp_tolerance_and_exact_rank,
    "full_rank": lambda: T.test_full_rank_blr_equals_dense_qr(32, 16, 4),
    "low_rank": lambda: T.test_exact_low_rank_blr_equals_dense_qr(96, 48, 8, 1),
    "qt_a": T.test_apply_q_roundtrip_and_qt_a_is_r,
    "lstsq": T.test_lstsq_matches_library_and_refinement,
    "metrics": T.test_metrics_measure_planted_errors,
    "blocked_full_rank": lambda: T.test_blocked_full_rank_equals_dense_qr(32, 16, 4),
    "blocked_low_rank": lambda: T.test_blocked_exact_low_rank_matches_dense_and_tiled(96, 48, 8, 1),
    "kernels": T.test_kernel_entries_closed_form,
    "rcb": T.test_rcb_order_leaves_and_boxes,
    "rcb_odd": lambda: [T.test_rcb_odd_leaf_count_and_anisotropic_box(s) for s in range(4)],
    "scale": T.test_ill_conditioned_scale,
    "column_scaling": T.test_column_scaling_is_a_right_diagonal_factor,
    "dense_threshold": T.test_dense_threshold_below_half_b,
    "admissibility": T.test_strong_admissibility_box_distance,
}

# (what the slip is, function, source text, replacement, pins that must fail)
MUTANTS = [
    ("reflector: beta takes the sign of alpha", "reflector",
     "beta = -norm if alpha >= 0.0 else norm", "beta = norm if alpha >= 0.0 else -norm", ["lapack"]),
    ("reflector: tau with the wrong sign", "reflector",
     "tau = (beta - alpha) / beta", "tau = (alpha - beta) / beta", ["reflector", "lapack", "full_rank"]),
    ("geqrt: tau dropped from the trailing update", "geqrt",
     "a[j:, j + 1:] -= tj * np.outer", "a[j:, j + 1:] -= np.outer", ["geqrt_wy", "full_rank"]),
    ("t_from_gram: sign of the recurrence", "t_from_gram",
     "= -tau[j] * (t[:j, :j]", "= tau[j] * (t[:j, :j]", ["geqrt_wy", "full_rank", "tsqrt"]),
    ("t_from_gram: transposed leading block", "t_from_gram",
     "(t[:j, :j] @ gram", "(t[:j, :j].T @ gram", ["geqrt_wy", "full_rank"]),
    ("larfb: T instead of T^T", "larfb", "(t.T @ (y.T @ c))", "(t @ (y.T @ c))", ["larfb", "full_rank"]),
    ("tsqrt: R row dropped from w", "tsqrt",
     "w = r[j, j + 1:] + y @ bv[:, j + 1:]", "w = y @ bv[:, j + 1:]", ["tsqrt", "full_rank"]),
    ("tsqrt: wrong sign on the R update", "tsqrt",
     "r[j, j + 1:] -= tj * w", "r[j, j + 1:] += tj * w", ["tsqrt", "full_rank"]),
    ("tpmqrt: T instead of T^T", "tpmqrt", "left_dense(t.T, s)", "left_dense(t, s)", ["tpmqrt", "full_rank"]),
    ("tpmqrt: S = R - Y^T A", "tpmqrt",
     "s = add(rkj, x, eps, cap)", "s = add(rkj, neg(x), eps, cap)", ["tpmqrt", "full_rank", "low_rank"]),
    ("tpmqrt: Y~ W not subtracted from A", "tpmqrt",
     "aij_new = add(aij, neg(mul(ytile, w)), eps, cap)", "aij_new = aij", ["tpmqrt", "full_rank"]),
    ("truncation_rank: one column too few", "truncation_rank",
     "return int(np.argmax(tail <= thresh))", "return max(0, int(np.argmax(tail <= thresh)) - 1)",
     ["truncation_rank", "rounded_addition"]),
    ("rounded_addition: sigma dropped from V", "rounded_addition",
     "qv @ (vt[:r].T * s[:r])", "qv @ vt[:r].T", ["rounded_addition", "low_rank"]),
    ("rounded_addition: B subtracted", "rounded_addition",
     "v = np.hstack([va, vb])", "v = np.hstack([va, -vb])", ["rounded_addition", "low_rank"]),
    ("compress_qrcp: tolerance ten times too loose", "compress_qrcp",
     "if tail <= eps * norm_a:", "if tail <= 10 * eps * norm_a:", ["compress"]),
    ("compress_qrcp: pivot on the smallest column", "compress_qrcp",
     "piv = r + int(np.argmax(col2))", "piv = r + int(np.argmin(col2))", ["compress"]),
    ("mul: transposed dense operand (OP3)", "mul",
     "v=y.d.T @ x.v", "v=y.d @ x.v", ["op3_op4", "tpmqrt"]),
    ("neg: both factors negated", "neg",
     'Tile("L", u=-x.u, v=x.v)', 'Tile("L", u=-x.u, v=-x.v)', ["tpmqrt", "low_rank"]),
    ("blr_qr: last tile row skipped", "blr_qr",
     "for i in range(k + 1, p):", "for i in range(k + 1, p - 1):", ["full_rank", "low_rank"]),
    ("blr_qr: LARFB skipped for low-rank R_kj", "blr_qr",
     'tl[k][j] = Tile("L", u=larfb(ykk, tkk, c.u), v=c.v)', "pass", ["low_rank"]),
    ("apply_qt: T instead of T^T", "apply_qt",
     "w = f.t[(i, k)].T @", "w = f.t[(i, k)] @", ["qt_a"]),
    ("apply_q: reflectors in factorization order", "apply_q",
     "for k in reversed(range(f.q)):", "for k in range(f.q):", ["qt_a"]),
    ("solve_r: diagonal division dropped", "_back_substitute",
     "x[i] /= r[i, i]", "pass", ["lstsq"]),
    ("solve_r: R_kj x_j added", "solve_r",
     "rhs -= t.u @ (t.v.T @ xj) if", "rhs += t.u @ (t.v.T @ xj) if", ["lstsq"]),
    ("residual: A compared with itself", "residual",
     "apply_q(f, rr) - a_dense", "a_dense - a_dense", ["metrics"]),
    ("residual: Q^T instead of Q", "residual", "apply_q(f, rr)", "apply_qt(f, rr)", ["metrics"]),
    ("orthogonality: Q Q^T instead of Q^T Q", "orthogonality",
     "q1.T @ q1 - np.eye(n)", "q1 @ q1.T - np.eye(q1.shape[0])", ["metrics", "low_rank"]),
    ("thin_q: Q^T [I; 0]", "thin_q", "return apply_q(f, e)", "return apply_qt(f, e)", ["metrics"]),
    ("block_column_qr: tau dropped from the update", "block_column_qr",
     "s[j:, j + 1:] -= tj * np.outer", "s[j:, j + 1:] -= np.outer", ["blocked_full_rank", "blocked_low_rank"]),
    ("block_column_qr: T from the wrong Gram matrix", "block_column_qr",
     "t_from_gram(y.T @ y, tau)", "t_from_gram(y @ y.T, tau)", ["blocked_full_rank", "blocked_low_rank"]),
    ("apply_block_column_reflector: T instead of T^T", "apply_block_column_reflector",
     "left_dense(t.T, s)", "left_dense(t, s)", ["blocked_full_rank", "blocked_low_rank"]),
    ("apply_block_column_reflector: one row of the sum dropped", "apply_block_column_reflector",
     "s = x if s is None else add(s, x, eps, cap)", "s = x", ["blocked_full_rank", "blocked_low_rank"]),
    ("compress: dense threshold ignored", "compress",
     "compress_qrcp(a, eps, out.cap)", "compress_qrcp(a, eps, b // 2)", ["dense_threshold"]),
    ("blr_qr: factorization ignores the dense threshold", "blr_qr",
     "p, q, b, cap = a.p, a.q, a.b, a.cap", "p, q, b, cap = a.p, a.q, a.b, a.b // 2", ["dense_threshold"]),
    ("compress: near tiles compressed", "compress",
     "if i == j or (inadmissible is not None and inadmissible[i][j]):", "if i == j:", ["admissibility"]),
    ("strong_admissibility: smaller diameter", "strong_admissibility",
     "diam = max(math.sqrt", "diam = min(math.sqrt", ["admissibility"]),
    ("strong_admissibility: gap from the box centres", "strong_admissibility",
     "gap = np.maximum(0.0, np.maximum(jlo - ihi, ilo - jhi))",
     "gap = np.abs((jlo + jhi) / 2 - (ilo + ihi) / 2)", ["admissibility"]),
    ("strong_admissibility: rows and columns swapped", "strong_admissibility",
     "bx, by = boxes(x, p), boxes(y, q)", "bx, by = boxes(x, q), boxes(y, p)", ["admissibility"]),
    # the seeded generators both sides take their inputs from
    ("kernel_entries: squared distance", "kernel_entries", "r = np.sqrt(diff2)", "r = diff2", ["kernels"]),
    ("kernel_entries: exp(+r)", "kernel_entries", "np.exp(-r)", "np.exp(r)", ["kernels"]),
    ("kernel_entries: rows scaled instead of columns", "kernel_entries",
     "a * col_scale[None, :]", "a * col_scale[:a.shape[0], None]", ["column_scaling"]),
    ("rcb_order: split along the shortest side", "rcb_order",
     "dim = int(np.argmax(ext))", "dim = int(np.argmin(ext))", ["rcb", "rcb_odd"]),
    ("rcb_order: floor(L/2) leaves to the left", "rcb_order",
     "int(math.ceil(leaves / 2)) * b", "(leaves // 2) * b", ["rcb_odd"]),
    ("rcb_order: leaf points not in original order", "rcb_order",
     "out.append(np.sort(ids))", "out.append(ids)", ["rcb"]),
    ("ill_conditioned_scale: divides by n", "ill_conditioned_scale",
     "np.arange(n) / (n - 1)", "np.arange(n) / n", ["scale"]),
    ("random_blr_dense: full-rank off-diagonal tiles", "random_blr_dense",
     "t = rng.standard_normal((b, k)) @ rng.standard_normal((b, k)).T", "t = rng.standard_normal((b, b))",
     ["low_rank"]),
]


def plant(monkeypatch, name, old, new):
    """Recompile oracle function `name` with `old` replaced by `new` and
    patch it into every oracle module that binds it."""
    mods = [m for m in (O, D, W) if name in vars(m)]
    original = getattr(mods[0], name)
    src = textwrap.dedent(inspect.getsource(original))
    assert src.count(old) == 1, f"{name}: planted text must occur exactly once"
    ns = dict(vars(inspect.getmodule(original)))
    exec(compile(src.replace(old, new), f"<mutant of {name}>", "exec"), ns)
    for m in mods:
        if getattr(m, name) is original:
            monkeypatch.setattr(m, name, ns[name])


@pytest.mark.parametrize("what,name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(monkeypatch, what, name, old, new, pins):
    plant(monkeypatch, name, old, new)
    survived = [p for p in pins if not _fails(PINS[p])]
    assert not survived, f"{what}: pins {survived} did not catch it"


def test_pins_pass_without_a_mistake():
    failing = [p for p, fn in PINS.items() if _fails(fn)]
    assert not failing, failing
