"""Conversions between the oracle's tiles and the library's tile layout
(test infrastructure)."""
import numpy as np

from oracle import blr_qr as O


def oracle_to_lib(a: O.BLRMatrix):
    """(ranks (p*q,), tiles (p*q*b*b,)) in the library layout of a BLR matrix."""
    p, q, b = a.p, a.q, a.b
    cap = b // 2
    ranks = np.empty(p * q, dtype=np.int32)
    tiles = np.zeros(p * q * b * b)
    for j in range(q):
        for i in range(p):
            t = a.tiles[i][j]
            off = (j * p + i) * b * b
            blk = tiles[off:off + b * b]
            if t.kind == "D":
                ranks[j * p + i] = -1
                blk[:] = t.d.ravel(order="F")
            else:
                r = t.rank
                ranks[j * p + i] = r
                blk[:b * r] = t.u.ravel(order="F")
                blk[b * cap:b * cap + b * r] = t.v.ravel(order="F")
    return ranks, tiles


def lib_tile(ranks, tiles, p, b, i, j):
    """Tile (i,j) as an oracle Tile."""
    cap = b // 2
    off = (j * p + i) * b * b
    blk = tiles[off:off + b * b]
    r = int(ranks[j * p + i])
    if r < 0:
        return O.Tile("D", d=blk.reshape(b, b, order="F").copy())
    u = blk[:b * r].reshape(b, r, order="F").copy()
    v = blk[b * cap:b * cap + b * r].reshape(b, r, order="F").copy()
    return O.Tile("L", u=u, v=v)


def lib_to_oracle(ranks, tiles, p, q, b) -> O.BLRMatrix:
    return O.BLRMatrix(p, q, b, [[lib_tile(ranks, tiles, p, b, i, j) for j in range(q)]
                                 for i in range(p)])


def lib_r_dense(ranks, tiles, p, q, b):
    """n x n upper triangular R of a factor's in-place storage."""
    n = q * b
    r = np.zeros((n, n))
    for k in range(q):
        for j in range(k, q):
            t = lib_tile(ranks, tiles, p, b, k, j).dense()
            if j == k:
                t = np.triu(t)
            r[k * b:(k + 1) * b, j * b:(j + 1) * b] = t
    return r


def lib_y_dense(ranks, tiles, p, b, i, k):
    """Y~_ik (i > k) densified, or Y_kk (unit lower) for i == k."""
    t = lib_tile(ranks, tiles, p, b, i, k).dense()
    if i == k:
        return np.tril(t, -1) + np.eye(b)
    return t


def tiles_of(a, b):
    return lambda i, j: a[i * b:(i + 1) * b, j * b:(j + 1) * b]
