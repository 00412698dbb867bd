"""Pins for the oracle's symmetric SpMM, dense expansion, norm and CSB tile store."""
import numpy as np
import pytest

import oracle
from conftest import golden_path


def random_upper(n, density, rng, integer=False):
    mask = np.triu(rng.random((n, n)) < density, 1) | np.eye(n, dtype=bool)
    r, c = np.nonzero(mask)
    if integer:
        v = rng.integers(-8, 9, len(r)).astype(np.float64)
    else:
        v = rng.standard_normal(len(r))
    return oracle.Coo(n, r, c, v)


def dense_by_indexing(H):
    """Full symmetric matrix built independently of the oracle with numpy indexing."""
    A = np.zeros((H.n, H.n))
    A[H.rows, H.cols] = H.vals
    A[H.cols, H.rows] = H.vals
    return A


@pytest.mark.parametrize("n,nb", [(1, 1), (7, 3), (50, 8), (300, 16)])
def test_spmm_integer_exact(n, nb):
    """Small integers: every partial sum is exact in FP64, so the product must equal the
    dense product exactly (special case reducing to a library matmul)."""
    rng = np.random.default_rng(n * 31 + nb)
    H = random_upper(n, 0.2, rng, integer=True)
    X = rng.integers(-8, 9, (n, nb)).astype(np.float64)
    Y = oracle.spmm(H, X)
    assert np.array_equal(Y, dense_by_indexing(H) @ X)


def test_spmm_unit_vectors_reproduce_columns():
    rng = np.random.default_rng(3)
    H = random_upper(40, 0.3, rng)
    A = dense_by_indexing(H)
    Y = oracle.spmm(H, np.eye(40))
    assert np.array_equal(Y, A)
    assert np.array_equal(oracle.dense(H), A)


def test_spmm_symmetry_identity():
    """X^T (H Z) = (H X)^T Z for symmetric H."""
    rng = np.random.default_rng(4)
    H = random_upper(120, 0.1, rng)
    X = rng.standard_normal((120, 5))
    Z = rng.standard_normal((120, 4))
    lhs = X.T @ oracle.spmm(H, Z)
    rhs = oracle.spmm(H, X).T @ Z
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


def test_norm_inf():
    rng = np.random.default_rng(5)
    H = random_upper(60, 0.2, rng)
    A = dense_by_indexing(H)
    assert oracle.norm_inf(H) == pytest.approx(np.abs(A).sum(axis=1).max(), rel=1e-14)


def read_tiles_golden():
    out = {}
    for line in open(golden_path("tiles_5x5_b2.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, rest = line.split(None, 1)
        if key == "entries":
            out[key] = [[float(x) for x in e.split()] for e in rest.split("|")]
        else:
            out[key] = [float(x) for x in rest.split()]
    return out


def test_tiles_golden_5x5():
    g = read_tiles_golden()
    e = np.array(g["entries"])
    H = oracle.Coo(5, e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), e[:, 2])
    T = oracle.tiles(H, b=2)
    assert T["ntiles"] == 6
    assert T["tile_rowptr"].tolist() == [int(x) for x in g["tile_rowptr"]]
    assert T["tile_col"].tolist() == [int(x) for x in g["tile_col"]]
    assert T["tile_ptr"].tolist() == [int(x) for x in g["tile_ptr"]]
    assert T["rc"].tolist() == [int(x) for x in g["rc"]]
    assert T["v64"].tolist() == g["vals"]


@pytest.mark.parametrize("n,b", [(1, 256), (300, 256), (1000, 64), (513, 256)])
def test_tiles_roundtrip(n, b):
    rng = np.random.default_rng(n + b)
    H = random_upper(n, 0.05, rng)
    perm = rng.permutation(H.nnz)
    Hp = oracle.Coo(n, H.rows[perm], H.cols[perm], H.vals[perm])
    T = oracle.tiles(Hp, b)
    nt = (n + b - 1) // b
    rp, tc, tp, rc = T["tile_rowptr"], T["tile_col"], T["tile_ptr"], T["rc"]
    assert rp[0] == 0 and rp[-1] == T["ntiles"] and len(rp) == nt + 1
    assert tp[0] == 0 and tp[-1] == H.nnz
    rows, cols, vals = [], [], []
    for tr in range(nt):
        assert np.all(np.diff(tc[rp[tr]:rp[tr + 1]]) > 0)  # tiles sorted by column, unique
        for t in range(rp[tr], rp[tr + 1]):
            assert tc[t] >= tr  # upper triangle of tiles
            seg = rc[tp[t]:tp[t + 1]]
            assert len(seg) > 0 and np.all(np.diff(seg.astype(np.int64)) > 0)  # (r, c) order
            r = (seg >> 16).astype(np.int64) + tr * b
            c = (seg & 0xFFFF).astype(np.int64) + int(tc[t]) * b
            rows += r.tolist(); cols += c.tolist(); vals += T["v64"][tp[t]:tp[t + 1]].tolist()
    back = np.array(rows) * n + np.array(cols)
    orig = H.rows * n + H.cols
    o1 = np.argsort(back); o2 = np.argsort(orig)
    assert np.array_equal(back[o1], orig[o2])
    assert np.array_equal(np.array(vals)[o1], H.vals[o2])
    assert np.array_equal(T["v32"], T["v64"].astype(np.float32))


def test_tiles_rejects_bad_input():
    ok = oracle.Coo(4, [0, 1], [1, 3], [1.0, 2.0])
    oracle.tiles(ok, 2)
    with pytest.raises(ValueError, match="below"):
        oracle.tiles(oracle.Coo(4, [2], [1], [1.0]), 2)
    with pytest.raises(ValueError, match="duplicate"):
        oracle.tiles(oracle.Coo(4, [0, 0], [1, 1], [1.0, 1.0]), 2)
    with pytest.raises(ValueError, match="range"):
        oracle.tiles(oracle.Coo(4, [0], [4], [1.0]), 2)
