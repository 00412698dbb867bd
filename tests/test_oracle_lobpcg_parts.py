"""Pins for the oracle's pieces of one LOBPCG iteration: block inner product, linear
combination, block-diagonal preconditioner (eq. 11), Rayleigh-Ritz (eq. 9), and the
paper's initial-guess statements of Section 3.3.1 (eqs. 12, 13)."""
import numpy as np
import pytest

import oracle
from test_oracle_sparse import dense_by_indexing, random_upper


def test_gram_and_lincomb_integer_exact():
    rng = np.random.default_rng(11)
    A = rng.integers(-8, 9, (500, 7)).astype(np.float64)
    B = rng.integers(-8, 9, (500, 5)).astype(np.float64)
    C = rng.integers(-8, 9, (7, 4)).astype(np.float64)
    assert np.array_equal(oracle.gram(A, B), A.T @ B)
    assert np.array_equal(oracle.lincomb(A, C), A @ C)


def test_block_precond_bp1_is_jacobi():
    """With 1x1 blocks, eq. 11 reduces to w_ij = r_ij / (h_ii - mu_j)."""
    rng = np.random.default_rng(12)
    H = random_upper(50, 0.2, rng)
    A = dense_by_indexing(H)
    mu = np.array([-3.0, 0.5, 7.0])
    R = rng.standard_normal((50, 3))
    W = oracle.block_precond(H, oracle.uniform_bounds(50, 1), mu, R)
    expect = R / (np.diag(A)[:, None] - mu[None, :])
    assert np.abs(W - expect).max() <= 1e-14 * np.abs(expect).max()


@pytest.mark.parametrize("n,bp", [(64, 32), (70, 32), (100, 7)])
def test_block_precond_solves_each_block(n, bp):
    rng = np.random.default_rng(n + bp)
    H = random_upper(n, 0.3, rng)
    A = dense_by_indexing(H)
    mu = np.array([0.1, -2.0])
    R = rng.standard_normal((n, 2))
    bounds = oracle.uniform_bounds(n, bp)
    W = oracle.block_precond(H, bounds, mu, R)
    for i in range(len(bounds) - 1):
        s = slice(bounds[i], bounds[i + 1])
        blk = A[s, s]
        for j in range(2):
            res = (blk - mu[j] * np.eye(blk.shape[0])) @ W[s, j] - R[s, j]
            assert np.linalg.norm(res) <= 1e-11 * np.abs(blk).sum() * max(np.linalg.norm(W[s, j]), 1.0)


def test_rayleigh_ritz_recovers_eigenpairs():
    rng = np.random.default_rng(13)
    n = 80
    H = random_upper(n, 0.2, rng)
    A = dense_by_indexing(H)
    w, Z = oracle.syev(A)
    Y = Z[:, :6] @ np.linalg.qr(rng.standard_normal((6, 6)))[0] * 3.0  # non-orthonormal basis of the span
    theta, C = oracle.rayleigh_ritz(Y.T @ A @ Y, Y.T @ Y)
    assert np.abs(theta - w[:6]).max() <= 1e-12 * np.abs(w).max()
    assert np.abs(C.T @ (Y.T @ Y) @ C - np.eye(6)).max() <= 1e-12


def test_rayleigh_ritz_interlacing_random_subspace():
    """Ritz values from an m-dimensional subspace bound the eigenvalues from above:
    theta_i >= lambda_i (Courant-Fischer), and G C = M C Theta."""
    rng = np.random.default_rng(14)
    n, m = 100, 9
    H = random_upper(n, 0.15, rng)
    A = dense_by_indexing(H)
    w, _ = oracle.syev(A)
    Y = rng.standard_normal((n, m))
    G, M = Y.T @ A @ Y, Y.T @ Y
    theta, C = oracle.rayleigh_ritz(G, M)
    assert np.all(theta >= w[:m] - 1e-10)
    assert np.all(theta <= w[-m:] + 1e-10)
    assert np.abs(G @ C - M @ C * theta).max() <= 1e-9 * np.abs(G).max()


def test_rayleigh_ritz_rejects_singular_gram():
    Y = np.zeros((10, 2))
    Y[0] = 1.0  # two identical columns: Y^T Y = [[1, 1], [1, 1]], last pivot exactly 0
    with pytest.raises(np.linalg.LinAlgError):
        oracle.rayleigh_ritz(Y.T @ Y, Y.T @ Y)


def two_level(n1, n2, eps, rng):
    """Symmetric H = [[H11, eps*H21^T], [eps*H21, H22]] with H22's spectrum well above H11's."""
    n = n1 + n2
    A = np.zeros((n, n))
    B = rng.standard_normal((n1, n1)); A[:n1, :n1] = B + B.T
    D = rng.standard_normal((n2, n2)); A[n1:, n1:] = D + D.T + 40.0 * np.eye(n2)
    C = rng.standard_normal((n2, n1)); A[n1:, :n1] = eps * C; A[:n1, n1:] = eps * C.T
    r, c = np.nonzero(np.triu(A) != 0)
    return oracle.Coo(n, r, c, A[r, c]), A


def test_eq12_zero_padded_guess_residual_bound():
    """X0 = [X1; 0] with H11 X1 = X1 Theta1: r_j = H21 x_j and ||r_j|| <= ||H21|| (eq. 12)."""
    rng = np.random.default_rng(21)
    n1, n2 = 20, 60
    H, A = two_level(n1, n2, 0.3, rng)
    w1, Z1 = oracle.syev(A[:n1, :n1])
    X0 = np.zeros((n1 + n2, 4)); X0[:n1] = Z1[:, :4]
    R = oracle.spmm(H, X0) - X0 * w1[:4]
    assert np.abs(R[:n1]).max() <= 1e-12 * np.abs(A).max()
    assert np.allclose(R[n1:], A[n1:, :n1] @ Z1[:, :4], atol=1e-12)
    norm21 = np.linalg.norm(A[n1:, :n1], 2)
    assert np.all(np.linalg.norm(R, axis=0) <= norm21 * (1 + 1e-12))


def test_eq13_block_diag_precond_gives_correction_and_eps_squared():
    """With T_j = diag{H11, H22} - theta_j I applied to the eq.-12 residual, the paper states
    W0 = -[0; Y1] where Y1 solves the second block row exactly: Y1 = -(H22 - theta I)^{-1} H21 X1
    (Section 3.3.1). Then span{X0, W0} contains the eq.-13 guess, so one Rayleigh-Ritz step on it
    leaves a residual of order eps^2: halving the coupling quarters the residual."""
    rng = np.random.default_rng(22)
    n1, n2 = 16, 48
    res = []
    for eps in [0.02, 0.01, 0.005]:
        H, A = two_level(n1, n2, eps, np.random.default_rng(22))
        w1, Z1 = oracle.syev(A[:n1, :n1])
        x1, th = Z1[:, 0], w1[0]
        X0 = np.zeros((n1 + n2, 1)); X0[:n1, 0] = x1
        R = oracle.spmm(H, X0) - X0 * th
        # exact-arithmetic residual of eq. 12 is [0; H21 x1]; the first block is only rounding
        # noise, and H11 - theta I is singular there, so take the exact zero as the paper does
        R[:n1] = 0.0
        W0 = oracle.block_precond(H, np.array([0, n1, n1 + n2]), np.array([th]), R)
        Y1 = -np.linalg.solve(A[n1:, n1:] - th * np.eye(n2), A[n1:, :n1] @ x1)
        assert np.abs(W0[:n1]).max() <= 1e-13
        assert np.abs(W0[n1:, 0] + Y1).max() <= 1e-10 * np.abs(Y1).max()
        S = np.hstack([X0, W0])
        theta, C = oracle.rayleigh_ritz(S.T @ oracle.spmm(H, S), S.T @ S)
        x = S @ C[:, 0]
        r = oracle.spmm(H, x[:, None])[:, 0] - theta[0] * x
        res.append(np.linalg.norm(r) / np.linalg.norm(x))
    r1 = res[0] / res[1]
    r2 = res[1] / res[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, res


def _blocks(A, bounds):
    return [A[bounds[i]:bounds[i + 1], bounds[i]:bounds[i + 1]] for i in range(len(bounds) - 1)]


@pytest.mark.parametrize("bp", [5, 16, 256])
def test_krylov_one_step_closed_forms(bp):
    """One FOM step is w = (r^T r / r^T A r) r; one minimal-residual step is
    w = (r^T A r / ||A r||^2) r (A = H~_[i] - mu_j I)."""
    rng = np.random.default_rng(40 + bp)
    n = 3 * bp + 2
    H = random_upper(n, 0.4, rng)
    Ad = dense_by_indexing(H)
    bounds = oracle.uniform_bounds(n, bp)
    mu = np.array([-0.7, 0.3])
    R = rng.standard_normal((n, 2))
    Wf = oracle.block_krylov(H, bounds, mu, R, "fom", 1)
    Wm = oracle.block_krylov(H, bounds, mu, R, "minres", 1)
    for i, B in enumerate(_blocks(Ad, bounds)):
        s = slice(bounds[i], bounds[i + 1])
        for j in range(2):
            A = B - mu[j] * np.eye(B.shape[0])
            r = R[s, j]
            Ar = A @ r
            np.testing.assert_allclose(Wf[s, j], (r @ r) / (r @ Ar) * r, rtol=1e-11, atol=0)
            np.testing.assert_allclose(Wm[s, j], (r @ Ar) / (Ar @ Ar) * r, rtol=1e-11, atol=0)


@pytest.mark.parametrize("bp", [2, 3])
def test_krylov_full_space_is_the_direct_solve(bp):
    """With as many steps as the block order the Krylov space is the whole block space, so FOM
    and the minimal-residual iterate both equal the direct solve of eq. 11 (a 2-step process on
    2 x 2 blocks stops early on the invariant subspace)."""
    rng = np.random.default_rng(50 + bp)
    n = 7 * bp
    H = random_upper(n, 0.6, rng)
    bounds = oracle.uniform_bounds(n, bp)
    mu = np.array([0.25, -1.5, 2.0])
    R = rng.standard_normal((n, 3))
    Wd = oracle.block_precond(H, bounds, mu, R)
    for method in ("fom", "minres"):
        W = oracle.block_krylov(H, bounds, mu, R, method, 3)
        assert np.abs(W - Wd).max() <= 1e-9 * np.abs(Wd).max()


@pytest.mark.parametrize("steps", [2, 3])
@pytest.mark.parametrize("bp", [24, 256])
def test_krylov_galerkin_and_minimal_residual(steps, bp):
    """FOM: r - A w is orthogonal to K_s(A, r). Minimal residual: ||r - A w|| is no larger than
    for any other w in K_s(A, r) (checked against the FOM iterate and random members). Blocks of
    256 rows are whole diagonal tiles, the blocks of Section 4.3's preconditioner."""
    rng = np.random.default_rng(60 + steps + bp)
    n = 2 * bp
    H = random_upper(n, 0.3, rng)
    Ad = dense_by_indexing(H)
    bounds = oracle.uniform_bounds(n, bp)
    lam_all = np.linalg.eigvalsh(_blocks(Ad, bounds)[0])
    mu = np.array([lam_all[3] + 0.01, lam_all[0] - 1.0])  # one indefinite shift, one definite
    R = rng.standard_normal((n, 2))
    Wf = oracle.block_krylov(H, bounds, mu, R, "fom", steps)
    Wm = oracle.block_krylov(H, bounds, mu, R, "minres", steps)
    for i, B in enumerate(_blocks(Ad, bounds)):
        s = slice(bounds[i], bounds[i + 1])
        for j in range(2):
            A = B - mu[j] * np.eye(bp)
            r = R[s, j]
            K = np.stack([np.linalg.matrix_power(A, t) @ r for t in range(steps)], axis=1)
            res_f = r - A @ Wf[s, j]
            assert np.abs(K.T @ res_f).max() <= 1e-8 * np.abs(K).max() * np.linalg.norm(r)
            rm = np.linalg.norm(r - A @ Wm[s, j])
            assert rm <= np.linalg.norm(res_f) * (1 + 1e-10)
            for _ in range(20):
                w = K @ rng.standard_normal(steps)
                assert rm <= np.linalg.norm(r - A @ w) * (1 + 1e-10)


def test_krylov_abs_is_direct_below_the_spectrum_and_spd():
    rng = np.random.default_rng(70)
    n, bp = 60, 20
    H = random_upper(n, 0.3, rng)
    Ad = dense_by_indexing(H)
    bounds = oracle.uniform_bounds(n, bp)
    lo = min(np.linalg.eigvalsh(B).min() for B in _blocks(Ad, bounds))
    R = rng.standard_normal((n, 2))
    mu = np.array([lo - 0.5, lo - 3.0])
    Wa = oracle.block_krylov(H, bounds, mu, R, "abs")
    Wd = oracle.block_precond(H, bounds, mu, R)
    assert np.abs(Wa - Wd).max() <= 1e-10 * np.abs(Wd).max()
    mu2 = np.array([0.0, 0.4])  # inside the spectra: |A|^{-1} stays positive definite
    Wa2 = oracle.block_krylov(H, bounds, mu2, R, "abs")
    for i in range(len(bounds) - 1):
        s = slice(bounds[i], bounds[i + 1])
        for j in range(2):
            assert R[s, j] @ Wa2[s, j] > 0


# Eigenvalue offsets (from the shift) and start-vector weights in the eigenbasis for which the
# projected 2 x 2 tridiagonal of two Lanczos steps on (A, r) is exactly singular: with
# m_k = r^T A^k r = sum_i x_i^2 a_i^k, det T is proportional to m_1 m_3 - m_2^2, and
# a = (-1, 1, 2), x^2 = (1/11, 1, 1) give m_1 m_3 - m_2^2 = (32/11)(96/11) - (56/11)^2 = 0 while
# m_1 = 32/11 != 0 (the first pivot is fine).
BREAK2_A = np.array([-1.0, 1.0, 2.0])
BREAK2_X = np.array([1.0 / np.sqrt(11.0), 1.0, 1.0])
# Two eigen-directions with x^2 = (1/2, 1/2) and a = (-1, 1): r^T A r = 0, the one-step pivot.
BREAK1_A = np.array([-1.0, 1.0])
BREAK1_X = np.array([1.0, 1.0]) / np.sqrt(2.0)


def fom_breakdown_block(bp, mu, rng, coords, a, x, dense=False):
    """A bp x bp symmetric block B and a vector r such that A = B - mu I restricted to the
    Krylov space of r has the spectrum mu + a on the eigen-directions that r touches, with r's
    weights x. The other eigenvalues are mu + 3 + 0.5 i (well away). With dense=False only the
    rows in `coords` are coupled (a small rotation), so the block is sparse; with dense=True
    the whole block is rotated by a random orthogonal matrix."""
    k = len(coords)
    d = mu + 3.0 + 0.5 * np.arange(bp)
    d[coords] = mu + a
    if dense:
        Q = np.linalg.qr(rng.standard_normal((bp, bp)))[0]
        B = (Q * d) @ Q.T
        r = Q[:, coords] @ x
    else:
        Qk = np.linalg.qr(rng.standard_normal((k, k)))[0]
        B = np.diag(d)
        B[np.ix_(coords, coords)] = (Qk * (mu + a)) @ Qk.T
        r = np.zeros(bp)
        r[coords] = Qk @ x
    return (B + B.T) / 2, r


@pytest.mark.parametrize("dense", [False, True])
def test_krylov_fom_breakdown_falls_back_to_minimal_residual(dense):
    """The FOM breakdown rule of the oracle (a pivot of the projected tridiagonal below 1e-4 of
    its largest entry, Sections 3.2 and 4.3 leave the case open) made to fire, with results fixed
    by the mathematics and not by the oracle's own algorithm:
      - two steps on a vector whose 2 x 2 projected matrix is singular: FOM's iterate does not
        exist, and minimal residual stagnates (its residual cannot fall where FOM is undefined,
        for a symmetric A), so the fallback must return the one-step minimal-residual iterate
        (r^T A r / ||A r||^2) r -- the same vector that the 2 x 2 least-squares closed form over
        span{r, A r} gives;
      - three steps on the same vector: r lies in a 3-dimensional invariant subspace, so the
        minimal-residual iterate is the exact solve A^{-1} r, although the unpivoted elimination
        of the 3 x 3 tridiagonal meets the zero second pivot;
      - one step on it: the pivot r^T A r / r^T r is fine, and FOM gives (r^T r / r^T A r) r;
      - one step on a vector with r^T A r = 0: the fallback's iterate is 0."""
    rng = np.random.default_rng(90 + dense)
    bp, mu = 12, 5.0
    B, r2 = fom_breakdown_block(bp, mu, rng, [1, 4, 9], BREAK2_A, BREAK2_X, dense)
    B1, r1 = fom_breakdown_block(bp, mu, rng, [2, 7], BREAK1_A, BREAK1_X, dense)
    n = 2 * bp
    Hd = np.zeros((n, n))
    Hd[:bp, :bp] = B
    Hd[bp:, bp:] = B1
    iu = np.triu_indices(n)
    keep = Hd[iu] != 0.0
    H = oracle.Coo(n, iu[0][keep].astype(np.int64), iu[1][keep].astype(np.int64), Hd[iu][keep])
    R = np.zeros((n, 1))
    R[:bp, 0] = r2
    R[bp:, 0] = r1
    bounds = oracle.uniform_bounds(n, bp)
    A = B - mu * np.eye(bp)
    A1 = B1 - mu * np.eye(bp)
    Ar = A @ r2
    m = [r2 @ np.linalg.matrix_power(A, k) @ r2 for k in range(5)]
    assert abs(m[1] * m[3] - m[2] ** 2) <= 1e-12 * m[2] ** 2 and m[1] > 1.0
    c = np.linalg.solve(np.array([[m[2], m[3]], [m[3], m[4]]]), np.array([m[1], m[2]]))
    ls2 = c[0] * r2 + c[1] * Ar
    mr1 = (r2 @ Ar) / (Ar @ Ar) * r2
    np.testing.assert_allclose(ls2, mr1, rtol=1e-10, atol=1e-12)
    tol = 1e-10 * np.linalg.norm(r2)
    for method in ("fom", "minres"):
        W2 = oracle.block_krylov(H, bounds, [mu], R, method, 2)[:, 0]
        assert np.all(np.isfinite(W2))
        assert np.abs(W2[:bp] - mr1).max() <= tol
        W3 = oracle.block_krylov(H, bounds, [mu], R, method, 3)[:, 0]
        assert np.abs(W3[:bp] - np.linalg.solve(A, r2)).max() <= tol
    W1 = oracle.block_krylov(H, bounds, [mu], R, "fom", 1)[:, 0]
    np.testing.assert_allclose(W1[:bp], (r2 @ r2) / (r2 @ Ar) * r2, rtol=1e-11, atol=0)
    assert abs(r1 @ A1 @ r1) <= 1e-14
    assert np.abs(W1[bp:]).max() <= 1e-12 * np.linalg.norm(r1)
