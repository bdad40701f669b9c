"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *draws* inputs: point clouds, their ordering, and the
kernel-matrix entries those points define.  It holds none of the BLR-QR
arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method's code.

Workloads (the paper's own data sets are not available, these stand in):

* ``inv1d``      -- A(i,j) = 1/(|x_i - y_j| + 1e-3), x, y uniform on [0,1],
                    sorted ascending (a 1D integral-equation-like kernel).
* ``yukawa3d``   -- A(i,j) = exp(-r)/(r + 1e-3), r = |x_i - y_j|, x, y uniform
                    in [0,1]^3, ordered by recursive coordinate bisection.
                    Stands in for the spatial-statistics and BEM matrices of
                    Section 5 (dense kernel matrices with low-rank far field).
* ``laplace3d``  -- A(i,j) = 1/(r + 1e-3), same geometry.
* ``random``     -- the random BLR matrices of Section 5.1: dense N(0,1)
                    diagonal tiles, off-diagonal tiles X Y^T with X, Y b x k
                    N(0,1).

An optional column scaling d_j = 10^(-10 j/(n-1)) makes the ill-conditioned
variant (columns scaled by a geometric sequence from 1 to 1e-10).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KERNEL_IDS = {"inv1d": 0, "yukawa3d": 1, "laplace3d": 2}
KERNEL_DIM = {"inv1d": 1, "yukawa3d": 3, "laplace3d": 3}
KERNEL_DELTA = 1e-3  # regularisation added to the distance in every kernel


@dataclasses.dataclass
class KernelProblem:
    """A kernel matrix A(i,j) = K(|x_i - y_j|) * d_j on ordered point sets."""

    kernel: str
    x: np.ndarray          # (dim, m) float64, already ordered
    y: np.ndarray          # (dim, n) float64, already ordered
    b: int
    col_scale: np.ndarray | None = None  # (n,) or None

    @property
    def m(self) -> int:
        return self.x.shape[1]

    @property
    def n(self) -> int:
        return self.y.shape[1]

    @property
    def kernel_id(self) -> int:
        return KERNEL_IDS[self.kernel]

    def block(self, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
        """Entries A[r0:r1, c0:c1] in float64 (numpy, host)."""
        return kernel_entries(self.kernel, self.x[:, r0:r1], self.y[:, c0:c1],
                              None if self.col_scale is None else self.col_scale[c0:c1])

    def tile(self, i: int, j: int) -> np.ndarray:
        b = self.b
        return self.block(i * b, (i + 1) * b, j * b, (j + 1) * b)

    def dense(self) -> np.ndarray:
        return self.block(0, self.m, 0, self.n)


def kernel_entries(kernel: str, x: np.ndarray, y: np.ndarray,
                   col_scale: np.ndarray | None = None) -> np.ndarray:
    """K(|x_i - y_j|) for point arrays x (dim, m), y (dim, n)."""
    diff2 = np.zeros((x.shape[1], y.shape[1]))
    for d in range(x.shape[0]):
        diff2 += (x[d][:, None] - y[d][None, :]) ** 2
    r = np.sqrt(diff2)
    if kernel == "inv1d" or kernel == "laplace3d":
        a = 1.0 / (r + KERNEL_DELTA)
    elif kernel == "yukawa3d":
        a = np.exp(-r) / (r + KERNEL_DELTA)
    else:
        raise ValueError(f"unknown kernel {kernel!r}")
    if col_scale is not None:
        a = a * col_scale[None, :]
    return a


def rcb_order(pts: np.ndarray, b: int) -> np.ndarray:
    """Recursive coordinate bisection ordering of points (dim, N).

    Each split is along the longest side of the current bounding box, at the
    median; a node holding L leaves sends ceil(L/2) leaves of b points to the
    left.  Ties in the coordinate are broken by original index.  Inside a
    leaf, points keep ascending original index.  Returns the permutation.
    """
    n_pts = pts.shape[1]
    if n_pts % b != 0:
        raise ValueError("number of points must be a multiple of b")
    out: list[np.ndarray] = []
    stack = [np.arange(n_pts)]
    while stack:
        ids = stack.pop()
        leaves = len(ids) // b
        if leaves <= 1:
            out.append(np.sort(ids))
            continue
        sub = pts[:, ids]
        ext = sub.max(axis=1) - sub.min(axis=1)
        dim = int(np.argmax(ext))
        order = np.lexsort((ids, sub[dim]))
        n_left = int(math.ceil(leaves / 2)) * b
        left, right = ids[order[:n_left]], ids[order[n_left:]]
        stack.append(right)   # popped second
        stack.append(left)    # popped first: left subtree comes first
    return np.concatenate(out)


def ill_conditioned_scale(n: int) -> np.ndarray:
    """d_j = 10^(-10 j/(n-1)), j = 0..n-1: columns scaled from 1 to 1e-10."""
    if n == 1:
        return np.ones(1)
    return 10.0 ** (-10.0 * np.arange(n) / (n - 1))


def kernel_problem(kernel: str, m: int, n: int, b: int, seed_x: int, seed_y: int,
                   ill_conditioned: bool = False, extent=None) -> KernelProblem:
    """Seeded kernel-matrix workload.

    Points are uniform in the unit box, or in the box [0, extent[d]] per
    coordinate when extent is given (a stretched domain gives a small matrix
    the mix of near, mid and far tiles that the unit cube gives only at large
    sizes).  1D points are sorted ascending; 3D points are RCB-ordered with
    leaf size b.
    """
    dim = KERNEL_DIM[kernel]
    x = np.random.default_rng(seed_x).random((dim, m))
    y = np.random.default_rng(seed_y).random((dim, n))
    if extent is not None:
        e = np.asarray(extent, dtype=np.float64).reshape(dim, 1)
        x = x * e
        y = y * e
    if dim == 1:
        x = np.sort(x, axis=1)
        y = np.sort(y, axis=1)
    else:
        x = np.ascontiguousarray(x[:, rcb_order(x, b)])
        y = np.ascontiguousarray(y[:, rcb_order(y, b)])
    scale = ill_conditioned_scale(n) if ill_conditioned else None
    return KernelProblem(kernel, x, y, b, scale)


# Named workloads, sized as in the benchmark configurations.
def inv1d_2048x1024(b: int = 128) -> KernelProblem:
    """2048 x 1024, b = 128 (16 x 8 tiles), 1D inverse-distance kernel."""
    return kernel_problem("inv1d", 2048, 1024, b, 101, 102)


def yukawa3d(m: int, n: int, b: int = 512, seed_x: int = 301, seed_y: int = 302,
             ill_conditioned: bool = False) -> KernelProblem:
    return kernel_problem("yukawa3d", m, n, b, seed_x, seed_y, ill_conditioned)


def random_blr_dense(m: int, n: int, b: int, k: int, seed: int) -> np.ndarray:
    """Random BLR matrix of Section 5.1 as a dense array (small sizes only).

    Diagonal tiles (i == j) are N(0,1); every other tile is X Y^T with X, Y
    b x k N(0,1).  Drawn tile by tile in column-major tile order.
    """
    rng = np.random.default_rng(seed)
    p, q = m // b, n // b
    a = np.empty((m, n))
    for j in range(q):
        for i in range(p):
            if i == j:
                t = rng.standard_normal((b, b))
            else:
                t = rng.standard_normal((b, k)) @ rng.standard_normal((b, k)).T
            a[i * b:(i + 1) * b, j * b:(j + 1) * b] = t
    return a


def gaussian_rhs(m: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides B (m x nrhs), N(0,1)."""
    return np.random.default_rng(seed).standard_normal((m, nrhs))


def batched_laplace3d(count: int = 64, seed: int = 401) -> list:
    """The batched uneven workload: `count` independent problems, m drawn
    uniformly from {4096, 6144, ..., 16384} (seed), n = m / 2, Laplace
    kernel on 3D uniform points with per-problem seeds 4000 + 2 s and
    4001 + 2 s.  Returns (m, n, seed_x, seed_y) tuples; the points are drawn
    (and RCB-ordered for the chosen tile size) by kernel_problem."""
    sizes = np.arange(4096, 16384 + 1, 2048)
    ms = np.random.default_rng(seed).choice(sizes, size=count)
    return [(int(m), int(m) // 2, 4000 + 2 * s, 4001 + 2 * s) for s, m in enumerate(ms)]
