"""Plain FP64 CPU oracle of the tiled Householder BLR-QR (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  Slow on purpose:
every step is the paper's operation written out on whole tiles, in the order
the paper gives, with numpy's QR/SVD/matmul as the only library primitives.

What it follows (Apriansyah & Yokota, "Parallel QR Factorization of Block
Low-Rank Matrices"):

* BLR format, Eq. 7 (Section 3.1): tile (i,j) is dense, or U V^T with
  U, V of b x r; U has orthonormal columns because compression is a
  truncated rank-revealing QR (Section 3.1 and Section 5).
* Compression rank: smallest r with ||A_ij - U V^T||_F <= eps ||A_ij||_F
  (Section 3.1); tiles needing rank > b/2 stay dense (Section 3.1), or
  above a lower dense threshold given with the matrix.
* Strong admissibility (Section 3.1, eta): tiles whose row and column
  clusters are near stay dense (strong_admissibility).
* OP1..OP4 and the rounded addition of Algorithm 6 (Section 3.1).
* Tiled Householder QR, Algorithm 4, with the BLR tile kernels of
  Section 3.4: diagonal QR (3.4.1), apply block reflector (3.4.2), update QR
  on [R_kk; V^T] (3.4.3, Eq. 21) and apply trapezoidal block reflector
  (3.4.4), with a recompression after every low-rank sum (Section 3.1).
* Left multiplication by Q and Q^T in the tiled order (Algorithm 5, read
  with the "I -" that the printed update omits).
* The blocked (block-column) Householder BLR-QR of Section 3.3: Householder
  QR of each stacked block column of A^V blocks (Eqs. 13-17) and the
  block-column reflector applied to the columns on its right (Eq. 18).
* Res and Orth of Section 5.

Readings where the paper is silent (the same list is kept in the design
notes): Householder sign convention of LAPACK; Algorithm 6 truncates at the
smallest r whose Frobenius tail is <= eps times the norm of the sum itself;
a low-rank result whose rank exceeds the dense threshold (b/2 by default,
the value the paper names, or a lower one given with the matrix) is stored
dense (the exact sum);
a rank-0 tile is a valid low-rank tile with empty factors.

Pins: see tests/test_oracle.py.  The whole factorization is pinned to the
textbook dense QR (oracle/dense_qr.py) in the full-rank case; the tile
kernels to explicit dense reflector products; Algorithm 6 to its error bound
and orthonormality; compression to its defining tolerance and to
largest-norm pivoting; Res and Orth to closed forms on planted errors.
tests/test_oracle_mutations.py plants one-slip mistakes in these functions
and checks that the pins catch each of them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .dense_qr import reflector

# ----------------------------------------------------------------------------
# Tiles (Eq. 7)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Tile:
    """A BLR tile: kind 'D' with d (b x b), or kind 'L' with u, v (b x r)."""

    kind: str
    d: np.ndarray | None = None
    u: np.ndarray | None = None
    v: np.ndarray | None = None

    @property
    def rank(self) -> int:
        return -1 if self.kind == "D" else self.u.shape[1]

    def dense(self) -> np.ndarray:
        return self.d.copy() if self.kind == "D" else self.u @ self.v.T

    def copy(self) -> "Tile":
        if self.kind == "D":
            return Tile("D", d=self.d.copy())
        return Tile("L", u=self.u.copy(), v=self.v.copy())


def dense_tile(d: np.ndarray) -> Tile:
    return Tile("D", d=np.array(d, dtype=np.float64, copy=True))


def lr_tile(u: np.ndarray, v: np.ndarray) -> Tile:
    return Tile("L", u=np.array(u, dtype=np.float64, copy=True),
                v=np.array(v, dtype=np.float64, copy=True))


# ----------------------------------------------------------------------------
# Compression (Section 3.1; truncated rank-revealing QR as in Section 5)
# ----------------------------------------------------------------------------


def truncation_rank(sigma: np.ndarray, eps: float) -> int:
    """Smallest r with sqrt(sum_{l>=r} sigma_l^2) <= eps sqrt(sum sigma_l^2)."""
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    total = float(np.sum(s2))
    if total == 0.0:
        return 0
    tail = np.append(np.cumsum(s2[::-1])[::-1], 0.0)  # tail[r] = sum_{l>=r}
    thresh = (eps * math.sqrt(total)) ** 2
    return int(np.argmax(tail <= thresh))


def compress_qrcp(a: np.ndarray, eps: float, max_rank: int) -> Tile:
    """Truncated column-pivoted Householder QR of one tile.

    A P = Q R is built column by column (pivot = largest remaining column
    norm of the trailing block, first index on ties); it stops at the
    smallest r whose trailing block satisfies ||R22||_F <= eps ||A||_F, which
    is exactly ||A - Q_r R_r P^T||_F.  U = Q_r (orthonormal), V = P R_r^T.
    A tile that needs rank > max_rank is returned dense.
    """
    a0 = np.array(a, dtype=np.float64, copy=True)
    a = a0.copy()
    m, n = a.shape
    norm_a = float(np.linalg.norm(a))
    perm = np.arange(n)
    refl = []
    r = 0
    while True:
        tail = float(np.linalg.norm(a[r:, r:])) if r < min(m, n) else 0.0
        if tail <= eps * norm_a:
            break
        if r == max_rank:
            return dense_tile(a0)
        col2 = np.sum(a[r:, r:] ** 2, axis=0)
        piv = r + int(np.argmax(col2))
        if piv != r:
            a[:, [r, piv]] = a[:, [piv, r]]
            perm[[r, piv]] = perm[[piv, r]]
        beta, tau, v = reflector(a[r:, r])
        a[r:, r + 1:] -= tau * np.outer(v, v @ a[r:, r + 1:])
        a[r, r] = beta
        a[r + 1:, r] = 0.0
        refl.append((tau, v))
        r += 1
    # U = Q [I_r; 0]
    u = np.zeros((m, r))
    u[:r, :r] = np.eye(r)
    for j in reversed(range(r)):
        tau, v = refl[j]
        u[j:] -= tau * np.outer(v, v @ u[j:])
    v_fac = np.zeros((n, r))
    v_fac[perm, :] = a[:r, :].T           # V = P R_r^T
    return lr_tile(u, v_fac)


def compress_svd(a: np.ndarray, rank: int) -> Tile:
    """Best rank-`rank` approximation (truncated SVD): U = left vectors,
    V = right vectors times singular values."""
    uu, s, vt = np.linalg.svd(np.asarray(a, dtype=np.float64))
    return lr_tile(uu[:, :rank], vt[:rank].T * s[:rank])


@dataclasses.dataclass
class BLRMatrix:
    p: int
    q: int
    b: int
    tiles: list            # tiles[i][j]
    dense_rank: int = 0    # dense threshold; 0 (or anything outside [1, b/2]) means b/2

    @property
    def cap(self) -> int:
        """Largest rank a low-rank tile may have: a tile (or a rounded sum)
        that needs more is stored dense (Section 3.1's fallback, applied
        with the threshold b/2 the paper names, or a lower one)."""
        if 0 < self.dense_rank <= self.b // 2:
            return self.dense_rank
        return self.b // 2

    def dense(self) -> np.ndarray:
        b = self.b
        a = np.zeros((self.p * b, self.q * b))
        for i in range(self.p):
            for j in range(self.q):
                a[i * b:(i + 1) * b, j * b:(j + 1) * b] = self.tiles[i][j].dense()
        return a

    def copy(self) -> "BLRMatrix":
        return BLRMatrix(self.p, self.q, self.b,
                         [[t.copy() for t in row] for row in self.tiles], self.dense_rank)

    def ranks(self) -> np.ndarray:
        return np.array([[t.rank for t in row] for row in self.tiles])


def compress(tile_fn, p: int, q: int, b: int, eps: float = 0.0,
             fixed_rank: int = 0, dense_rank: int = 0, inadmissible=None) -> BLRMatrix:
    """BLR matrix: diagonal tiles dense (weak admissibility), and so is every
    tile (i,j) with inadmissible[i][j] true (strong admissibility, see
    strong_admissibility); every other tile compressed (fixed rank by
    truncated SVD, or tolerance eps by truncated QRCP; a tile that needs a
    rank above the dense threshold -- dense_rank, or b/2 when 0 -- falls back
    to dense)."""
    out = BLRMatrix(p, q, b, [], dense_rank)
    for i in range(p):
        row = []
        for j in range(q):
            a = tile_fn(i, j)
            if i == j or (inadmissible is not None and inadmissible[i][j]):
                row.append(dense_tile(a))
            elif fixed_rank > 0:
                row.append(compress_svd(a, fixed_rank))
            else:
                row.append(compress_qrcp(a, eps, out.cap))
        out.tiles.append(row)
    return out


def strong_admissibility(x: np.ndarray, y: np.ndarray, b: int, eta: float) -> np.ndarray:
    """Inadmissible (near) tiles under strong admissibility (Section 3.1,
    eta): the row cluster i is the points x[:, i b:(i+1) b], the column
    cluster j the points y[:, j b:(j+1) b]; tile (i,j) is near, and stays
    dense, when the distance between the two clusters' axis-aligned
    bounding boxes is below eta times the larger of the two box diameters.
    The paper names eta and says that a larger eta leaves more blocks
    inadmissible without printing a formula; this is the standard box
    criterion with that property.  Returns a p x q boolean array."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p, q = x.shape[1] // b, y.shape[1] // b

    def boxes(pts, n):
        return [(pts[:, c * b:(c + 1) * b].min(axis=1), pts[:, c * b:(c + 1) * b].max(axis=1))
                for c in range(n)]

    bx, by = boxes(x, p), boxes(y, q)
    near = np.zeros((p, q), dtype=bool)
    for i in range(p):
        ilo, ihi = bx[i]
        for j in range(q):
            jlo, jhi = by[j]
            gap = np.maximum(0.0, np.maximum(jlo - ihi, ilo - jhi))
            dist = math.sqrt(float(np.sum(gap * gap)))
            diam = max(math.sqrt(float(np.sum((ihi - ilo) ** 2))), math.sqrt(float(np.sum((jhi - jlo) ** 2))))
            near[i, j] = dist < eta * diam
    return near


# ----------------------------------------------------------------------------
# OP1..OP4 and Algorithm 6 (Section 3.1)
# ----------------------------------------------------------------------------


def rounded_addition(ua, va, ub, vb, eps: float, cap: int) -> Tile:
    """Algorithm 6: U = [U_A U_B], V = [V_A V_B]; QR both; SVD of R_U R_V^T;
    keep the first r_eps columns of Q_U u and of Q_V v sigma.  A result
    whose rank exceeds cap is stored dense (the exact sum)."""
    u = np.hstack([ua, ub])
    v = np.hstack([va, vb])
    b = u.shape[0]
    if u.shape[1] == 0:
        return lr_tile(np.zeros((b, 0)), np.zeros((v.shape[0], 0)))
    qu, ru = np.linalg.qr(u)
    qv, rv = np.linalg.qr(v)
    uu, s, vt = np.linalg.svd(ru @ rv.T)
    r = truncation_rank(s, eps)
    if r > cap:
        return dense_tile(u @ v.T)
    return lr_tile(qu @ uu[:, :r], qv @ (vt[:r].T * s[:r]))


def add(x: Tile, y: Tile, eps: float, cap: int) -> Tile:
    """OP1 (dense result when either operand is dense) or OP2 (rounded)."""
    if x.kind == "L" and y.kind == "L":
        return rounded_addition(x.u, x.v, y.u, y.v, eps, cap)
    return dense_tile(x.dense() + y.dense())


def neg(x: Tile) -> Tile:
    if x.kind == "D":
        return Tile("D", d=-x.d)
    return Tile("L", u=-x.u, v=x.v)


def transpose(x: Tile) -> Tile:
    if x.kind == "D":
        return Tile("D", d=x.d.T.copy())
    return Tile("L", u=x.v, v=x.u)


def mul(x: Tile, y: Tile) -> Tile:
    """OP3 (low-rank times dense) and OP4 (U_A (V_A^T U_B V_B^T))."""
    if x.kind == "L" and y.kind == "L":
        return Tile("L", u=x.u, v=y.v @ (y.u.T @ x.v))
    if x.kind == "L":
        return Tile("L", u=x.u, v=y.d.T @ x.v)
    if y.kind == "L":
        return Tile("L", u=x.d @ y.u, v=y.v)
    return Tile("D", d=x.d @ y.d)


def left_dense(m: np.ndarray, x: Tile) -> Tile:
    """M X for a dense matrix M (OP3 from the left)."""
    if x.kind == "L":
        return Tile("L", u=m @ x.u, v=x.v)
    return Tile("D", d=m @ x.d)


# ----------------------------------------------------------------------------
# Tile kernels (Section 3.4)
# ----------------------------------------------------------------------------


def t_from_gram(gram: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Compact-WY T (Eq. 3) from reflector Gram matrix G = Y^T Y and taus:
    T[j,j] = tau_j, T[:j,j] = -tau_j T[:j,:j] G[:j,j] (Schreiber & Van Loan)."""
    nb = len(tau)
    t = np.zeros((nb, nb))
    for j in range(nb):
        t[j, j] = tau[j]
        if j > 0:
            t[:j, j] = -tau[j] * (t[:j, :j] @ gram[:j, j])
    return t


def geqrt(a: np.ndarray):
    """QR of the dense diagonal tile (Section 3.4.1): A = (I - Y T Y^T) R.

    Returns R (upper triangular), Y (unit lower triangular), T (upper)."""
    a = np.array(a, dtype=np.float64, copy=True)
    b = a.shape[0]
    y = np.zeros((b, b))
    tau = np.zeros(b)
    for j in range(b):
        beta, tj, v = reflector(a[j:, j])
        a[j:, j + 1:] -= tj * np.outer(v, v @ a[j:, j + 1:])
        a[j, j] = beta
        a[j + 1:, j] = 0.0
        y[j:, j] = v
        tau[j] = tj
    return np.triu(a), y, t_from_gram(y.T @ y, tau)


def larfb(y: np.ndarray, t: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Q^T C with Q = I - Y T Y^T (Section 3.4.2)."""
    return c - y @ (t.T @ (y.T @ c))


def tsqrt(r: np.ndarray, bv: np.ndarray):
    """Update QR (Section 3.4.3): QR([R; B]) for upper triangular R (b x b)
    and B = V^T (r x b, low-rank tile) or the dense tile (b x b).

    Reflector j is [e_j; y_j]; returns R', Y (rows(B) x b, column j = y_j)
    and T with Q = I - [I; Y] T [I; Y]^T (Eq. 20)."""
    r = np.array(r, dtype=np.float64, copy=True)
    bv = np.array(bv, dtype=np.float64, copy=True)
    nb = r.shape[0]
    tau = np.zeros(nb)
    for j in range(nb):
        x = np.concatenate([[r[j, j]], bv[:, j]])
        beta, tj, v = reflector(x)
        y = v[1:]
        w = r[j, j + 1:] + y @ bv[:, j + 1:]
        r[j, j + 1:] -= tj * w
        bv[:, j + 1:] -= tj * np.outer(y, w)
        r[j, j] = beta
        bv[:, j] = y
        tau[j] = tj
    # [I; Y]^T [I; Y] = I + Y^T Y; off-diagonal entries come from Y alone.
    return r, bv, t_from_gram(bv.T @ bv, tau)


def tpmqrt(ytile: Tile, t: np.ndarray, rkj: Tile, aij: Tile, eps: float,
           cap: int) -> tuple[Tile, Tile]:
    """Apply trapezoidal block reflector (Section 3.4.4):

        [R_kj; A_ij] <- [R_kj; A_ij] - [I; Y~] T^T (R_kj + Y~^T A_ij)

    as BLR operations: S = R_kj + Y~^T A_ij (OP3/OP4 then OP1/OP2),
    W = T^T S (OP3), R_kj - W (OP1/OP2), A_ij - Y~ W (OP4 then OP1/OP2).
    Y~ = U_ik Y_ik is stored as the low-rank tile (U_ik, Y_ik^T), or dense."""
    x = mul(transpose(ytile), aij)
    s = add(rkj, x, eps, cap)
    w = left_dense(t.T, s)
    rkj_new = add(rkj, neg(w), eps, cap)
    aij_new = add(aij, neg(mul(ytile, w)), eps, cap)
    return rkj_new, aij_new


# ----------------------------------------------------------------------------
# Algorithm 4 on a BLR matrix
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Factor:
    """In-place BLR factor: tiles[k][k] holds R_kk (upper) and Y_kk (strictly
    lower, unit diagonal implied); tiles[k][j], j > k, hold R_kj; tiles[i][k],
    i > k, hold Y~_ik; t[(i, k)] holds T_ik (t[(k, k)] from the diagonal QR)."""

    p: int
    q: int
    b: int
    tiles: list
    t: dict

    def r_dense(self) -> np.ndarray:
        b, n = self.b, self.q * self.b
        r = np.zeros((n, n))
        for k in range(self.q):
            for j in range(k, self.q):
                blk = self.tiles[k][j].dense()
                if j == k:
                    blk = np.triu(blk)
                r[k * b:(k + 1) * b, j * b:(j + 1) * b] = blk
        return r

    def y_diag(self, k: int) -> np.ndarray:
        d = self.tiles[k][k].d
        return np.tril(d, -1) + np.eye(self.b)

    def y_dense(self, i: int, k: int) -> np.ndarray:
        return self.tiles[i][k].dense()

    def ranks(self) -> np.ndarray:
        return np.array([[t.rank for t in row] for row in self.tiles])


def blr_qr(a: BLRMatrix, eps: float) -> Factor:
    """Algorithm 4 with the BLR tile kernels of Section 3.4 (weak or strong
    admissibility: any tile may be dense; diagonal tiles are dense)."""
    p, q, b, cap = a.p, a.q, a.b, a.cap
    tl = [[t.copy() for t in row] for row in a.tiles]
    ts = {}
    for k in range(q):
        if tl[k][k].kind != "D":
            tl[k][k] = dense_tile(tl[k][k].dense())
        rkk, ykk, tkk = geqrt(tl[k][k].d)
        ts[(k, k)] = tkk
        for j in range(k + 1, q):
            c = tl[k][j]
            if c.kind == "L":
                tl[k][j] = Tile("L", u=larfb(ykk, tkk, c.u), v=c.v)
            else:
                tl[k][j] = dense_tile(larfb(ykk, tkk, c.d))
        for i in range(k + 1, p):
            aik = tl[i][k]
            bv = aik.v.T if aik.kind == "L" else aik.d
            rkk, yik, tik = tsqrt(rkk, bv)
            tl[i][k] = Tile("L", u=aik.u, v=yik.T.copy()) if aik.kind == "L" \
                else dense_tile(yik)
            ts[(i, k)] = tik
            for j in range(k + 1, q):
                tl[k][j], tl[i][j] = tpmqrt(tl[i][k], tik, tl[k][j], tl[i][j], eps, cap)
        tl[k][k] = dense_tile(np.triu(rkk) + np.tril(ykk, -1))
    return Factor(p, q, b, tl, ts)


# ----------------------------------------------------------------------------
# Blocked Householder BLR-QR (Section 3.3; Algorithm 2 on a BLR matrix)
# ----------------------------------------------------------------------------


def block_column_qr(col: list):
    """Triangularization of a block column (Section 3.3.1, Eqs. 13-17):
    Householder QR of the stacked A^V_ik (the dense block, or V^T of a
    low-rank block; the diagonal block is dense), i = k..p-1.

    Returns R_kk (b x b upper), the tails Y~_ik = A^U_ik Y_ik as tiles
    (low-rank (U_ik, Y_ik^T) where A_ik is low-rank, dense otherwise; the
    diagonal one unit lower triangular) and T_k (b x b upper) with
    Q_k = I - Y~ T_k Y~^T over the stacked rows of the column."""
    parts = [t.d if t.kind == "D" else t.v.T for t in col]
    rows = [p.shape[0] for p in parts]
    s = np.vstack(parts).astype(np.float64, copy=True)
    nb = s.shape[1]
    y = np.zeros_like(s)
    tau = np.zeros(nb)
    for j in range(nb):
        beta, tj, v = reflector(s[j:, j])
        s[j:, j + 1:] -= tj * np.outer(v, v @ s[j:, j + 1:])
        s[j, j] = beta
        s[j + 1:, j] = 0.0
        y[j:, j] = v
        tau[j] = tj
    t = t_from_gram(y.T @ y, tau)
    tails, r0 = [], 0
    for tile, nr in zip(col, rows):
        yi = y[r0:r0 + nr]
        tails.append(Tile("L", u=tile.u, v=yi.T.copy()) if tile.kind == "L" else dense_tile(yi))
        r0 += nr
    return np.triu(s[:nb]), tails, t


def apply_block_column_reflector(tails: list, t: np.ndarray, col: list, eps: float, cap: int) -> list:
    """Q_k^T applied to a block column (Section 3.3.2, Eq. 18):
    S = sum_i Y~_ik^T A_ij (products OP3/OP4, rounded additions),
    W = T_k^T S, A_ij <- A_ij - Y~_ik W (each difference a rounded addition)."""
    s = None
    for yt, a in zip(tails, col):
        x = mul(transpose(yt), a)
        s = x if s is None else add(s, x, eps, cap)
    w = left_dense(t.T, s)
    return [add(a, neg(mul(yt, w)), eps, cap) for yt, a in zip(tails, col)]


@dataclasses.dataclass
class BlockedFactor:
    """Blocked factor: r[k][j] (j >= k) the tiles of R; y[k] the tails of
    block column k (rows k..p-1); t[k] its T_k."""

    p: int
    q: int
    b: int
    r: dict
    y: list
    t: list

    def r_dense(self) -> np.ndarray:
        b, n = self.b, self.q * self.b
        out = np.zeros((n, n))
        for (k, j), tile in self.r.items():
            out[k * b:(k + 1) * b, j * b:(j + 1) * b] = np.triu(tile.dense()) if j == k else tile.dense()
        return out

    def y_stacked(self, k: int) -> np.ndarray:
        """Y~ of block column k as a dense (m - k b) x b matrix."""
        return np.vstack([yt.dense() for yt in self.y[k]])


def blr_qr_blocked(a: BLRMatrix, eps: float) -> BlockedFactor:
    """Blocked Householder BLR-QR: for each block column, triangularize it
    (block_column_qr), then apply its reflector to every block column on
    its right (apply_block_column_reflector)."""
    p, q, b, cap = a.p, a.q, a.b, a.cap
    tl = [[t.copy() for t in row] for row in a.tiles]
    r, ys, ts = {}, [], []
    for k in range(q):
        col = [tl[i][k] for i in range(k, p)]
        if col[0].kind != "D":
            col[0] = dense_tile(col[0].dense())
        rkk, tails, tk = block_column_qr(col)
        r[(k, k)] = dense_tile(rkk)
        ys.append(tails)
        ts.append(tk)
        for j in range(k + 1, q):
            new = apply_block_column_reflector(tails, tk, [tl[i][j] for i in range(k, p)], eps, cap)
            for i, tile in zip(range(k, p), new):
                tl[i][j] = tile
            r[(k, j)] = tl[k][j]
    return BlockedFactor(p, q, b, r, ys, ts)


def blocked_apply_qt(f: BlockedFactor, c: np.ndarray) -> np.ndarray:
    """Q^T C for the blocked factor, block columns in order."""
    b = f.b
    c = np.array(c, dtype=np.float64, copy=True)
    for k in range(f.q):
        yk = f.y_stacked(k)
        c[k * b:] -= yk @ (f.t[k].T @ (yk.T @ c[k * b:]))
    return c


def blocked_apply_q(f: BlockedFactor, c: np.ndarray) -> np.ndarray:
    """Q C for the blocked factor, block columns in reverse order."""
    b = f.b
    c = np.array(c, dtype=np.float64, copy=True)
    for k in reversed(range(f.q)):
        yk = f.y_stacked(k)
        c[k * b:] -= yk @ (f.t[k] @ (yk.T @ c[k * b:]))
    return c


# ----------------------------------------------------------------------------
# Algorithm 5: left multiplication by Q^T and Q (exact, stored reflectors)
# ----------------------------------------------------------------------------


def apply_qt(f: Factor, c: np.ndarray) -> np.ndarray:
    """Q^T C, reflectors in factorization order."""
    b = f.b
    c = np.array(c, dtype=np.float64, copy=True)
    for k in range(f.q):
        ck = slice(k * b, (k + 1) * b)
        c[ck] = larfb(f.y_diag(k), f.t[(k, k)], c[ck])
        for i in range(k + 1, f.p):
            ci = slice(i * b, (i + 1) * b)
            yt = f.y_dense(i, k)
            w = f.t[(i, k)].T @ (c[ck] + yt.T @ c[ci])
            c[ck] -= w
            c[ci] -= yt @ w
    return c


def apply_q(f: Factor, c: np.ndarray) -> np.ndarray:
    """Q C, reflectors in reverse order (Algorithm 5 with the 'I -')."""
    b = f.b
    c = np.array(c, dtype=np.float64, copy=True)
    for k in reversed(range(f.q)):
        ck = slice(k * b, (k + 1) * b)
        for i in reversed(range(k + 1, f.p)):
            ci = slice(i * b, (i + 1) * b)
            yt = f.y_dense(i, k)
            w = f.t[(i, k)] @ (c[ck] + yt.T @ c[ci])
            c[ck] -= w
            c[ci] -= yt @ w
        y = f.y_diag(k)
        c[ck] = c[ck] - y @ (f.t[(k, k)] @ (y.T @ c[ck]))
    return c


# ----------------------------------------------------------------------------
# Least squares with the BLR R (QR used for least squares, Section 1)
# ----------------------------------------------------------------------------


def solve_r(f: Factor, c: np.ndarray) -> np.ndarray:
    """x with R x = c (block back substitution, R_kj low-rank or dense)."""
    b, q = f.b, f.q
    x = np.zeros((q * b,) + c.shape[1:])
    for k in reversed(range(q)):
        rhs = np.array(c[k * b:(k + 1) * b], copy=True)
        for j in range(k + 1, q):
            t = f.tiles[k][j]
            xj = x[j * b:(j + 1) * b]
            rhs -= t.u @ (t.v.T @ xj) if t.kind == "L" else t.d @ xj
        rkk = np.triu(f.tiles[k][k].d)
        x[k * b:(k + 1) * b] = _back_substitute(rkk, rhs)
    return x


def _back_substitute(r: np.ndarray, c: np.ndarray) -> np.ndarray:
    x = np.array(c, dtype=np.float64, copy=True)
    nb = r.shape[0]
    for i in reversed(range(nb)):
        if i + 1 < nb:
            x[i] -= r[i, i + 1:] @ x[i + 1:]
        x[i] /= r[i, i]
    return x


def blr_matvec(a: BLRMatrix, x: np.ndarray) -> np.ndarray:
    b = a.b
    y = np.zeros((a.p * b,) + x.shape[1:])
    for i in range(a.p):
        for j in range(a.q):
            t = a.tiles[i][j]
            xj = x[j * b:(j + 1) * b]
            y[i * b:(i + 1) * b] += t.u @ (t.v.T @ xj) if t.kind == "L" else t.d @ xj
    return y


def lstsq(f: Factor, bmat: np.ndarray, a: BLRMatrix | None = None,
          refine_steps: int = 0) -> np.ndarray:
    """x = R^{-1} (Q^T B)[:n]; optional refinement x += R^{-1} Q_1^T (B - A x)."""
    n = f.q * f.b
    x = solve_r(f, apply_qt(f, bmat)[:n])
    for _ in range(refine_steps):
        res = bmat - blr_matvec(a, x)
        x = x + solve_r(f, apply_qt(f, res)[:n])
    return x


# ----------------------------------------------------------------------------
# Accuracy metrics (Section 5)
# ----------------------------------------------------------------------------


def thin_q(f: Factor) -> np.ndarray:
    m, n = f.p * f.b, f.q * f.b
    e = np.zeros((m, n))
    e[:n, :n] = np.eye(n)
    return apply_q(f, e)


def residual(f: Factor, a_dense: np.ndarray) -> float:
    """||Q_1 R - A||_F / ||A||_F."""
    m, n = a_dense.shape
    rr = np.zeros((m, n))
    rr[:n] = f.r_dense()
    return float(np.linalg.norm(apply_q(f, rr) - a_dense) / np.linalg.norm(a_dense))


def orthogonality(f: Factor) -> float:
    """||Q_1^T Q_1 - I||_F / sqrt(n)."""
    q1 = thin_q(f)
    n = q1.shape[1]
    return float(np.linalg.norm(q1.T @ q1 - np.eye(n)) / math.sqrt(n))
