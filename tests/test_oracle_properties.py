"""Property checks of the oracle over random shapes (hypothesis): tile
counts from a single tile to tall ragged grids, tile sizes, ranks from 0 to
b/2, dense off-diagonal tiles.  Each drawn case must satisfy what Algorithm 4
and Section 5 fix whatever the shape: exact-rank inputs give the dense QR's
R (up to row signs), Q^T A = [R; 0], an orthogonal Q, and an R whose
diagonal tiles are upper triangular."""
import numpy as np
import pytest

from oracle import blr_qr as O
from oracle import dense_qr as D

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def _blr(rng, p, q, b, k, dense_frac):
    a = np.zeros((p * b, q * b))
    for j in range(q):
        for i in range(p):
            if i == j or rng.random() < dense_frac:
                t = rng.standard_normal((b, b)) + (3 * np.eye(b) if i == j else 0)
            else:
                t = rng.standard_normal((b, k)) @ rng.standard_normal((b, k)).T
            a[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
    return a


@hyp.settings(max_examples=60, deadline=None, derandomize=True)
@hyp.given(q=st.integers(1, 4), extra=st.integers(0, 4), b=st.sampled_from([4, 6, 8]),
           k=st.integers(0, 3), dense_frac=st.sampled_from([0.0, 0.3]), seed=st.integers(0, 2 ** 31 - 1))
def test_tiled_qr_properties_on_random_shapes(q, extra, b, k, dense_frac, seed):
    p = q + extra
    k = min(k, b // 2)
    rng = np.random.default_rng(seed)
    a = _blr(rng, p, q, b, k, dense_frac)
    blr = O.compress(lambda i, j: a[i * b:(i + 1) * b, j * b:(j + 1) * b], p, q, b, eps=1e-14)
    f = O.blr_qr(blr, 1e-15)
    m, n = p * b, q * b
    r = f.r_dense()
    scale = np.linalg.norm(a)
    # R: upper triangular, the dense QR's R up to row signs
    assert np.allclose(r, np.triu(r), atol=0.0)
    r_ref = np.linalg.qr(a, mode="r")
    assert np.linalg.norm(D.sign_normalize(r) - D.sign_normalize(r_ref)) <= 1e-11 * scale
    # Q^T A = [R; 0] and Q orthogonal (Section 5's Orth)
    qta = O.apply_qt(f, a)
    assert np.linalg.norm(qta[:n] - r) <= 1e-11 * scale
    assert np.linalg.norm(qta[n:]) <= 1e-11 * scale
    assert O.orthogonality(f) <= 1e-13
    assert O.residual(f, a) <= 1e-12
