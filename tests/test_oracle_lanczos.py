"""Pins for the oracle's Lanczos (full reorthogonalisation) against the dense solver."""
import numpy as np
import pytest

import oracle


def test_lanczos_matches_dense_c1(c1_problem, c1_dense_eig):
    H = c1_problem["H"]
    w, Z = c1_dense_eig
    k = 8
    lam, X, steps, conv = oracle.lanczos(H, k, 1e-12, c1_problem["normH"])
    assert conv
    rel = np.abs(lam - w[:k]) / np.maximum(np.abs(w[:k]), 1.0)
    assert rel.max() <= 1e-10
    res = oracle.residual_norms(H, X, lam)
    assert res.max() <= 1e-10 * c1_problem["normH"]
    for j in range(k):
        assert abs(abs(X[:, j] @ Z[:, j]) - 1.0) <= 1e-8


def random_sparse_sym(n, per_row, rng):
    rows, cols = [], []
    for i in range(n):
        js = rng.integers(0, n, per_row)
        for j in js:
            a, b = min(i, j), max(i, j)
            rows.append(a); cols.append(b)
    rows += list(range(n)); cols += list(range(n))
    key = np.unique(np.array(rows, dtype=np.int64) * n + np.array(cols, dtype=np.int64))
    r, c = key // n, key % n
    v = rng.standard_normal(len(r))
    v[r == c] = rng.uniform(0, 50, n)
    return oracle.Coo(n, r, c, v)


@pytest.mark.slow
def test_lanczos_matches_dense_random_n2000():
    rng = np.random.default_rng(2000)
    H = random_sparse_sym(2000, 5, rng)
    w, _ = oracle.syev(oracle.dense(H))
    lam, X, steps, conv = oracle.lanczos(H, 6, 1e-12)
    assert conv
    rel = np.abs(lam - w[:6]) / np.maximum(np.abs(w[:6]), 1.0)
    assert rel.max() <= 1e-10


def test_csr_forms_match_coo_forms_exactly(c1_problem, c1_dense_eig):
    """The CSR product and Lanczos (32-bit columns, used for the ~1e9-entry workload) visit the
    entries in the order of the generator's (row, col)-sorted COO, so they must equal the COO
    forms bit for bit; the Lanczos eigenvalues are then pinned to the dense solver as above."""
    H = c1_problem["H"]
    Hc = oracle.Csr.from_sorted_coo(H.n, H.rows, H.cols, H.vals)
    X = np.random.default_rng(5).standard_normal((H.n, 3))
    assert np.array_equal(oracle.spmm_csr(Hc, X), oracle.spmm(H, X))
    lam, Xl, steps, conv = oracle.lanczos(H, 5, 1e-12, c1_problem["normH"])
    lam_c, Xc, steps_c, conv_c = oracle.lanczos_csr(Hc, 5, 1e-12, c1_problem["normH"])
    assert conv and conv_c and steps == steps_c
    assert np.array_equal(lam, lam_c) and np.array_equal(Xl, Xc)
    w, _ = c1_dense_eig
    assert (np.abs(lam_c - w[:5]) / np.maximum(np.abs(w[:5]), 1.0)).max() <= 1e-10


def test_csr_product_on_random_matrix():
    rng = np.random.default_rng(11)
    H = random_sparse_sym(300, 7, rng)
    Hc = oracle.Csr.from_sorted_coo(H.n, H.rows, H.cols, H.vals)
    X = rng.standard_normal((300, 4))
    assert np.abs(oracle.spmm_csr(Hc, X) - oracle.dense(H) @ X).max() <= 1e-12 * np.abs(X).max() * 50
