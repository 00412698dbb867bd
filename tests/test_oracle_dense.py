"""Pins for the oracle's dense eigensolvers (Householder + QL, cyclic Jacobi) and the
tridiagonal QL, against closed forms, constructed spectra and invariants."""
import numpy as np
import pytest

import oracle
from conftest import golden_path

U = np.finfo(np.float64).eps


def householder_Q(n, rng, reflectors=6):
    """Orthogonal Q as a product of seeded Householder reflectors I - 2 u u^T."""
    Q = np.eye(n)
    for _ in range(reflectors):
        u = rng.standard_normal(n)
        u /= np.linalg.norm(u)
        Q = Q - 2.0 * np.outer(Q @ u, u)
    return Q


@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 200])
def test_known_spectrum(n):
    rng = np.random.default_rng(100 + n)
    d = rng.uniform(-10, 10, n)
    Q = householder_Q(n, rng)
    A = Q @ np.diag(d) @ Q.T
    A = 0.5 * (A + A.T)
    w, Z = oracle.syev(A)
    tol = 50 * n * U * np.abs(d).max()
    assert np.abs(w - np.sort(d)).max() <= tol
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-13 * max(n, 1)
    assert np.abs(A @ Z - Z * w).max() <= tol


def read_2x2():
    rows = []
    for line in open(golden_path("closed_forms_2x2.txt")):
        line = line.split("#")[0].split()
        if line:
            rows.append([float(x) for x in line])
    return np.array(rows)


@pytest.mark.parametrize("solver", ["ql", "jacobi"])
def test_closed_form_2x2_blocks(solver):
    g = read_2x2()
    m = len(g)
    A = np.zeros((2 * m, 2 * m))
    for i, (a, b, c, _, _) in enumerate(g):
        A[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[a, b], [b, c]]
    expect = np.sort(g[:, 3:5].ravel())
    w, _ = oracle.syev(A) if solver == "ql" else oracle.jacobi(A)
    assert np.abs(w - expect).max() <= 1e-13 * np.abs(expect).max()


def test_diagonal_matrix():
    d = np.array([3.0, -1.0, 2.5, 0.0, -7.25, 2.5])
    w, Z = oracle.syev(np.diag(d))
    assert np.array_equal(w, np.sort(d))
    assert np.allclose(np.abs(Z), np.abs(Z).round())  # permutation matrix (up to sign)


@pytest.mark.parametrize("n", [3, 40, 120])
def test_trace_and_frobenius_invariants(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, _ = oracle.syev(A)
    assert abs(w.sum() - np.trace(A)) <= 1e-12 * n * np.abs(A).max()
    assert abs((w * w).sum() - (A * A).sum()) <= 1e-12 * (A * A).sum()


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64])
def test_jacobi_matches_ql(n):
    """Two independent algorithms agree to 1e-12 ||A|| (brute-force pin at n <= 64)."""
    rng = np.random.default_rng(7 * n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w1, Z1 = oracle.syev(A)
    w2, Z2 = oracle.jacobi(A)
    nrm = np.abs(A).sum(axis=1).max()
    assert np.abs(w1 - w2).max() <= 1e-12 * nrm
    assert np.abs(A @ Z2 - Z2 * w2).max() <= 1e-12 * nrm
    # eigenvectors agree up to sign where eigenvalues are separated
    gaps = np.diff(w1)
    for j in range(n):
        left = gaps[j - 1] if j > 0 else np.inf
        right = gaps[j] if j < n - 1 else np.inf
        if min(left, right) > 1e-6 * nrm:
            assert abs(abs(Z1[:, j] @ Z2[:, j]) - 1.0) <= 1e-9


@pytest.mark.parametrize("m", [1, 2, 10, 257])
def test_tridiagonal_laplacian_closed_form(m):
    """tridiag(-1, 2, -1) of order m: eigenvalues 2 - 2 cos(k pi/(m+1)), eigenvectors
    proportional to sin(j k pi/(m+1))."""
    d = 2.0 * np.ones(m)
    e = -np.ones(m - 1)
    w, Z = oracle.tridiag_eig(d, e)
    k = np.arange(1, m + 1)
    expect = 2 - 2 * np.cos(k * np.pi / (m + 1))
    assert np.abs(w - expect).max() <= 1e-13 * 4
    j = np.arange(1, m + 1)
    for kk in [1, m]:
        s = np.sin(j * kk * np.pi / (m + 1))
        s /= np.linalg.norm(s)
        assert abs(abs(s @ Z[:, kk - 1]) - 1.0) <= 1e-10


def test_gershgorin_containment(c1_problem, c1_dense_eig):
    """Every eigenvalue lies in the union of Gershgorin discs; here simply in
    [min(h_ii - r_i), max(h_ii + r_i)]."""
    H = c1_problem["H"]
    A = oracle.dense(H)
    dia = np.diag(A)
    rad = np.abs(A).sum(axis=1) - np.abs(dia)
    w, _ = c1_dense_eig
    assert w.min() >= (dia - rad).min() - 1e-9
    assert w.max() <= (dia + rad).max() + 1e-9
    assert np.abs(w).max() <= c1_problem["normH"] + 1e-9
