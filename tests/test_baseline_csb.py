"""The threaded CPU CSB SpMM baseline (the paper's CPU organisation of the product, Section 4.4)
against the oracle's plain COO product. FP32 values and FP32 products inside a tile, so the
bound is a few FP32 roundings of |H| |X| per row."""
import numpy as np
import pytest

import baseline
import oracle
import synth


def _abs_bound(n, r, c, v, X):
    """Row sums of |H| |X| over the full symmetric matrix."""
    A = np.zeros((n, X.shape[1]))
    ax = np.abs(X)
    np.add.at(A, r, np.abs(v)[:, None] * ax[c])
    off = r != c
    np.add.at(A, c[off], np.abs(v[off])[:, None] * ax[r[off]])
    return A


@pytest.mark.parametrize("nb", [1, 8, 16])
def test_csb_matches_oracle_c1(nb):
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    X = np.random.default_rng(nb).standard_normal((L.n, nb))
    M = baseline.CsbMatrix(L.n, r, c, v)
    Y = M.spmm(X)
    Yr = oracle.spmm(oracle.Coo(L.n, r, c, v), X)
    assert np.all(np.abs(Y - Yr) <= 1e-5 * _abs_bound(L.n, r, c, v, X) + 1e-300)


@pytest.mark.parametrize("threads", [1, 3])
def test_csb_ragged_tiles_and_threads(threads):
    # n not a multiple of the tile, entries in the last partial tile, a lone diagonal tile row
    rng = np.random.default_rng(7)
    n = 1000
    i = rng.integers(0, n, 6000)
    j = rng.integers(0, n, 6000)
    r = np.minimum(i, j)
    c = np.maximum(i, j)
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    key, idx = np.unique(r * n + c, return_index=True)
    r, c = r[idx], c[idx]
    v = rng.standard_normal(len(r))
    X = rng.standard_normal((n, 5))
    M = baseline.CsbMatrix(n, r, c, v, b=256)
    assert M.ntiles > 0
    Y = M.spmm(X, threads=threads)
    Yr = oracle.spmm(oracle.Coo(n, r, c, v), X)
    assert np.all(np.abs(Y - Yr) <= 1e-5 * _abs_bound(n, r, c, v, X) + 1e-300)


def test_csb_rejects_lower_and_duplicates():
    with pytest.raises(ValueError):
        baseline.CsbMatrix(4, np.array([1]), np.array([0]), np.array([1.0]))
    with pytest.raises(ValueError):
        baseline.CsbMatrix(4, np.array([0, 0]), np.array([1, 1]), np.array([1.0, 2.0]))
