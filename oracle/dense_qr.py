"""Textbook unblocked Householder QR (test infrastructure only).

Independent of the BLR oracle on purpose: this is the plain dense method of
Section 2.2 (A = QR, Eq. 1, computed one Householder reflection per column,
as in Golub & Van Loan's Householder QR), used to pin the BLR oracle in the
cases where the BLR factorization must reproduce dense QR exactly.

Reflector convention: for a column x with head alpha and tail norm sigma,
beta = -sign(alpha) ||x|| (sign(0) = +1), tau = (beta - alpha)/beta,
v = x / (alpha - beta) with v[0] = 1; a zero tail gives tau = 0.
"""
from __future__ import annotations

import numpy as np


def reflector(x: np.ndarray) -> tuple[float, float, np.ndarray]:
    """(beta, tau, v) with (I - tau v v^T) x = beta e_1 and v[0] = 1."""
    alpha = float(x[0])
    sigma = float(np.sqrt(np.sum(x[1:] ** 2)))
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return alpha, 0.0, v
    norm = float(np.hypot(alpha, sigma))
    beta = -norm if alpha >= 0.0 else norm
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return beta, tau, v


def householder_qr(a: np.ndarray) -> tuple[np.ndarray, list[tuple[float, np.ndarray]]]:
    """Unblocked Householder QR of a (m x n, m >= n).

    Returns R (n x n upper triangular) and the reflectors [(tau_j, v_j)],
    v_j of length m - j acting on rows j..m-1.
    """
    a = np.array(a, dtype=np.float64, copy=True)
    m, n = a.shape
    if m < n:
        raise ValueError("m >= n required")
    refl = []
    for j in range(n):
        beta, tau, v = reflector(a[j:, j])
        a[j:, j + 1:] -= tau * np.outer(v, v @ a[j:, j + 1:])
        a[j, j] = beta
        a[j + 1:, j] = 0.0
        refl.append((tau, v))
    return np.triu(a[:n, :]), refl


def apply_q(refl, c: np.ndarray) -> np.ndarray:
    """Q c for Q = H_0 H_1 ... H_{n-1} (applied right to left)."""
    c = np.array(c, dtype=np.float64, copy=True)
    for j in reversed(range(len(refl))):
        tau, v = refl[j]
        c[j:] -= tau * np.outer(v, v @ c[j:])
    return c


def apply_qt(refl, c: np.ndarray) -> np.ndarray:
    """Q^T c."""
    c = np.array(c, dtype=np.float64, copy=True)
    for j in range(len(refl)):
        tau, v = refl[j]
        c[j:] -= tau * np.outer(v, v @ c[j:])
    return c


def thin_q(refl, m: int, n: int) -> np.ndarray:
    """Q_1 = Q [I_n; 0] (m x n)."""
    e = np.zeros((m, n))
    e[:n, :n] = np.eye(n)
    return apply_q(refl, e)


def sign_normalize(r: np.ndarray) -> np.ndarray:
    """D R with D = diag(sign(diag R)) so that diag(D R) >= 0."""
    d = np.where(np.diag(r) < 0.0, -1.0, 1.0)
    return d[:, None] * r
