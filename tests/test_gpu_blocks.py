"""The pieces of one LOBPCG iteration on the GPU against the oracle: block inner product and
linear combination (Section 4.4) in FP64 and double-float, the block-diagonal preconditioner
(eq. 11) and the Rayleigh-Ritz step (eq. 9)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import random_upper

pytestmark = pytest.mark.gpu


def t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mode", ["fp64", "mixed", "tc"])
@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (1000, 16, 16), (4097, 48, 48), (3000, 8, 100), (20000, 49, 17)])
def test_gram_integer_exact(mode, n, p, q):
    if mode == "tc" and q > 64:
        pytest.skip("the tensor-core kernel takes p, q <= 64")
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n + p + q)
    A = rng.integers(-8, 9, (n, p)).astype(np.float64)
    B = rng.integers(-8, 9, (n, q)).astype(np.float64)
    G = lob.gram(t(A), t(B), mode).cpu().numpy()
    assert np.array_equal(G, oracle.gram(A, B))


@pytest.mark.parametrize("mode,rel", [("fp64", 4.0 * 2.0 ** -53), ("mixed", 2.0 ** -44)])
def test_gram_random_bound(mode, rel):
    """|G - G*| <= c n u |A|^T |B| with c = 4 (FP64) and a double-float unit of 2^-44."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(1)
    n = 200_000
    A = rng.standard_normal((n, 48)); B = rng.standard_normal((n, 48)) * 1e3
    G = lob.gram(t(A), t(B), mode).cpu().numpy()
    ref = oracle.gram(A, B)
    bound = np.abs(A).T @ np.abs(B) * rel * np.sqrt(n) * 4
    assert np.all(np.abs(G - ref) <= bound)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "tc"])
@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (5000, 48, 16), (4097, 32, 16), (1000, 7, 5), (129, 64, 16),
                                   (257, 65, 16), (300, 96, 40)])
def test_lincomb_exact_and_bound(mode, n, p, q):
    if mode == "tc" and p > 64:
        pytest.skip("the tensor-core kernel takes p, q <= 64")
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n * 3 + p)
    A = rng.integers(-8, 9, (n, p)).astype(np.float64)
    C = rng.integers(-8, 9, (p, q)).astype(np.float64)
    assert np.array_equal(lob.lincomb(t(A), t(C), mode).cpu().numpy(), oracle.lincomb(A, C))
    A = rng.standard_normal((n, p)); C = rng.standard_normal((p, q))
    Y = lob.lincomb(t(A), t(C), mode).cpu().numpy()
    rel = 2 * p * 2.0 ** -53 if mode == "fp64" else 2.0 ** -44 * p
    if mode == "tc":  # scaling groups: rows of A, columns of C (see test_lincomb_tensor_cores)
        ra = np.abs(A).max(axis=1, keepdims=True)
        cc = np.abs(C).max(axis=0, keepdims=True)
        bnd = 2.0 ** -44 * (np.abs(A) @ np.abs(C) + ra * np.abs(C).sum(axis=0, keepdims=True)
                            + np.abs(A).sum(axis=1, keepdims=True) * cc)
        assert np.all(np.abs(Y - oracle.lincomb(A, C)) <= bnd + 1e-300)
        return
    assert np.all(np.abs(Y - oracle.lincomb(A, C)) <= rel * (np.abs(A) @ np.abs(C)) + 1e-300)


@pytest.mark.parametrize("bp", [1, 32, 64])
def test_precond_matches_block_solve(bp):
    """FP32 arithmetic (footnote 5). The bound, derived to first order:
      - the S sweeps of FP32 cyclic Jacobi give H~ + E = Q diag(lambda) Q^T with Q orthogonal to
        ||Q^T Q - I|| <= c_J b_p u32 and ||E|| <= c_J b_p u32 ||H~||, c_J about the sweep count
        (each sweep touches every entry with b_p - 1 rotations of relative error ~u32);
      - (H~ + E - mu)^{-1} - (H~ - mu)^{-1} ~ -(H~ - mu)^{-1} E (H~ - mu)^{-1}, so E costs
        c_J b_p u32 kappa_j relative, kappa_j = ||H~|| / min |lambda - mu_j| over the blocks;
      - the apply w = Q f(lambda - mu) Q^T r adds two length-b_p FP32 products, 2 b_p u32 kappa_j.
    With c_J <= 14 (this matrix family converges in 6-10 sweeps): 16 b_p u32 kappa_j. Measured on
    the GPU, max err / (b_p u32 kappa_j) = 1.9 (b_p = 1), 6.0 (32), 7.7 (64)."""
    import paper_1609_01689_gb300 as lob
    L = synth.layout(3000, 7, 40, 4)
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    M = lob.Matrix(L.n, r, c, v, precond_block=bp)
    rng = np.random.default_rng(bp)
    R = rng.standard_normal((L.n, 8))
    mu = np.array([-5.0, -3.3, 4.9, 15.1, 24.7, 36.0, 45.2, 200.0])
    W = M.precond_apply(t(mu), t(R)).cpu().numpy()
    ref = oracle.block_precond(H, oracle.uniform_bounds(L.n, bp), mu, R)
    err = np.abs(W - ref).max(axis=0) / np.abs(ref).max(axis=0)
    bounds = oracle.uniform_bounds(L.n, bp)
    A = oracle.dense(H)
    kappa = np.ones(8)
    for i in range(len(bounds) - 1):
        lam_b = np.linalg.eigvalsh(A[bounds[i]:bounds[i + 1], bounds[i]:bounds[i + 1]])
        d = np.abs(lam_b[:, None] - mu[None, :])
        kappa = np.maximum(kappa, np.abs(lam_b).max() / d.min(axis=0))
    assert np.all(err <= 16 * bp * 2.0 ** -24 * kappa), (err, kappa)


@pytest.mark.parametrize("solve,steps", [("fom", 1), ("fom", 2), ("fom", 3), ("minres", 1), ("minres", 2),
                                         ("minres", 3), ("abs", 1)])
@pytest.mark.parametrize("bp", [32, 64])
def test_precond_krylov_matches_oracle(solve, steps, bp):
    """The Krylov solves of eq. 11 run in each block's FP32 eigenbasis on the GPU and by dense
    Lanczos in FP64 in the oracle (independent algorithms for the same iterate). Shifts below
    every block's spectrum (definite systems) for FOM / minimal residual, inside it for the
    absolute-value solve. The FP32 eigendecomposition carries the same error as for the direct
    solve (c_J b_p u32 kappa_j with c_J <= 14, see test_precond_matches_block_solve), and the
    iterate is a fixed low-degree rational function of the projected quantities, formed with two
    length-b_p FP32 products, so the same bound holds: 16 b_p u32 kappa_j, kappa_j =
    ||H~|| / min|lambda - mu_j|. Measured on the GPU, max err / (b_p u32 kappa_j) <= 3.4."""
    import paper_1609_01689_gb300 as lob
    L = synth.layout(2500, 7, 40, 5)
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    M = lob.Matrix(L.n, r, c, v, precond_block=bp)
    bounds = oracle.uniform_bounds(L.n, bp)
    A = oracle.dense(H)
    blocks = [np.linalg.eigvalsh(A[bounds[i]:bounds[i + 1], bounds[i]:bounds[i + 1]]) for i in range(len(bounds) - 1)]
    lo = min(b.min() for b in blocks)
    if solve == "abs":
        mu = np.array([-0.3, 4.1, 15.2, 33.3])
    else:
        mu = np.array([lo - 0.5, lo - 2.0, lo - 7.0, lo - 20.0])
    rng = np.random.default_rng(bp + steps)
    R = rng.standard_normal((L.n, 4))
    W = M.precond_apply(t(mu), t(R), solve=solve, steps=steps).cpu().numpy()
    guard = 1e-8 * oracle.norm_inf(H)
    ref = oracle.block_krylov(H, bounds, mu, R, solve, steps, guard)
    err = np.abs(W - ref).max(axis=0) / np.abs(ref).max(axis=0)
    kappa = np.ones(4)
    for lam_b in blocks:
        d = np.abs(lam_b[:, None] - mu[None, :])
        kappa = np.maximum(kappa, np.abs(lam_b).max() / d.min(axis=0))
    assert np.all(err <= 16 * bp * 2.0 ** -24 * kappa), (err, kappa)


def test_precond_bp1_is_jacobi_formula():
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(3)
    H = random_upper(700, 0.02, rng)
    H.vals[H.rows == H.cols] += 10.0
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals, precond_block=1)
    R = rng.standard_normal((700, 4))
    mu = np.array([0.5, -1.0, 2.0, 30.0])
    W = M.precond_apply(t(mu), t(R)).cpu().numpy()
    dia = np.zeros(700); dia[H.rows[H.rows == H.cols]] = H.vals[H.rows == H.cols]
    expect = R / (dia[:, None] - mu[None, :])
    assert np.abs(W - expect).max() <= 1e-6 * np.abs(expect).max()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [1, 8, 24, 48, 96])
def test_rayleigh_ritz_matches_oracle(m, mode):
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(m)
    Y = rng.standard_normal((400, m))
    A = oracle.dense(random_upper(400, 0.05, rng))
    G, Mm = Y.T @ A @ Y, Y.T @ Y
    th, C = lob.rayleigh_ritz(t(G), t(Mm), mode)
    th, C = th.cpu().numpy(), C.cpu().numpy()
    th_ref, _ = oracle.rayleigh_ritz(G, Mm)
    scale = np.abs(th_ref).max()
    assert np.abs(th - th_ref).max() <= 1e-11 * scale
    assert np.abs(C.T @ Mm @ C - np.eye(m)).max() <= 1e-10
    assert np.abs(G @ C - Mm @ C * th).max() <= 1e-10 * np.abs(G).max()


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_rayleigh_ritz_reports_indefinite(mode):
    import paper_1609_01689_gb300 as lob
    Mm = np.array([[1.0, 1.0], [1.0, 1.0]])
    with pytest.raises(np.linalg.LinAlgError):
        lob.rayleigh_ritz(t(np.eye(2)), t(Mm), mode)


@pytest.mark.parametrize("solve,steps", [("fom", 1), ("fom", 2), ("fom", 3), ("minres", 2), ("minres", 3)])
@pytest.mark.parametrize("ncol", [4, 20])
def test_precond_tiles_match_oracle(solve, steps, ncol):
    """Eq. 11 on the diagonal tiles (Section 4.3), the blocks being whole 256-row tiles: Krylov
    steps on the sparse tile in FP32 on the GPU, dense Lanczos in FP64 in the oracle. The last
    tile is partial (n = 2,500), and 20 columns take two passes of the kernel. Shifts below every
    tile's spectrum (definite systems). No eigendecomposition is involved: each Lanczos quantity
    (a tile-row product of at most b terms, a dot product of b terms) carries a relative error of
    at most gamma_b ~ b u32, and the s-step projected solve passes a perturbation of its
    coefficients on with a factor of at most kappa_j = ||H~|| / min |lambda - mu_j| over the tiles,
    so to first order the error is at most (s + 1) b u32 kappa_j <= 4 b u32 kappa_j (b = 256).
    Measured on the GPU, max err / (b u32 kappa_j) <= 0.009."""
    import paper_1609_01689_gb300 as lob
    L = synth.layout(2500, 7, 40, 5)
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    M = lob.Matrix(L.n, r, c, v, precond_block=256)
    bounds = oracle.uniform_bounds(L.n, 256)
    A = oracle.dense(H)
    blocks = [np.linalg.eigvalsh(A[bounds[i]:bounds[i + 1], bounds[i]:bounds[i + 1]]) for i in range(len(bounds) - 1)]
    lo = min(b.min() for b in blocks)
    mu = lo - np.array([0.5, 2.0, 7.0, 20.0] * 5)[:ncol]
    rng = np.random.default_rng(ncol + steps)
    R = rng.standard_normal((L.n, ncol))
    W = M.precond_apply(t(mu), t(R), solve=solve, steps=steps).cpu().numpy()
    ref = oracle.block_krylov(H, bounds, mu, R, solve, steps)
    err = np.abs(W - ref).max(axis=0) / np.abs(ref).max(axis=0)
    kappa = np.ones(ncol)
    for lam_b in blocks:
        d = np.abs(lam_b[:, None] - mu[None, :])
        kappa = np.maximum(kappa, np.abs(lam_b).max() / d.min(axis=0))
    assert np.all(err <= 4 * 256 * 2.0 ** -24 * kappa), (err, kappa)


def test_precond_tiles_rejects_what_it_cannot_do():
    """Tile mode needs FP32 values and takes only the Krylov solves, in lob_precond_apply and in a
    served request alike."""
    import paper_1609_01689_gb300 as lob
    L = synth.layout(1000, 6, 30, 2)
    r, c, v = synth.generate(L)
    with pytest.raises(lob.LobError):
        lob.Matrix(L.n, r, c, v, precond_block=256, values=lob.VALUES_FP64)
    with pytest.raises(lob.LobError):
        lob.Matrix(L.n, r, c, v, precond_block=100)
    M = lob.Matrix(L.n, r, c, v, precond_block=256)
    R = np.random.default_rng(1).standard_normal((L.n, 4))
    with pytest.raises(lob.LobError):
        M.precond_apply(t(np.zeros(4) - 9.0), t(R), solve="direct")
    srv = lob.Server(budget_bytes=1 << 30)
    with pytest.raises(lob.LobError):
        srv.submit(M, 2, 4, 1e-8, precond=True, precond_solve="direct")
    srv.submit(M, 2, 4, 1e-8, precond=True)  # FOM on the tiles is served
    srv.close()


def _breakdown_matrix(bp, nblk, mu, dense, seed):
    """Block-diagonal H whose even blocks make two-step FOM break down for column 0 and whose
    odd blocks make one-step FOM break down for column 1 (constructions and closed forms in
    test_oracle_lobpcg_parts); those columns are zero in the other blocks, and columns 2-3 are
    random. Every block's spectrum sits at mu - 1 and above."""
    from test_oracle_lobpcg_parts import BREAK1_A, BREAK1_X, BREAK2_A, BREAK2_X, fom_breakdown_block
    rng = np.random.default_rng(seed)
    n = bp * nblk
    Hd = np.zeros((n, n))
    R = rng.standard_normal((n, 4))
    c2 = [1, bp // 2, bp - 2]
    c1 = [3, bp - 1]
    for b in range(nblk):
        s = slice(b * bp, (b + 1) * bp)
        B2, r2 = fom_breakdown_block(bp, mu, rng, c2, BREAK2_A, BREAK2_X, dense)
        B1, r1 = fom_breakdown_block(bp, mu, rng, c1, BREAK1_A, BREAK1_X, dense)
        Hd[s, s] = B2 if b % 2 == 0 else B1
        R[s, 0] = r2 if b % 2 == 0 else 0.0
        R[s, 1] = r1 if b % 2 == 1 else 0.0
    # a few couplings between blocks: the preconditioner must ignore them
    for _ in range(3 * nblk):
        i, j = sorted(rng.integers(0, n, 2))
        if i // bp != j // bp:
            Hd[i, j] = Hd[j, i] = 0.25
    iu = np.triu_indices(n)
    keep = Hd[iu] != 0.0
    H = oracle.Coo(n, iu[0][keep].astype(np.int64), iu[1][keep].astype(np.int64), Hd[iu][keep])
    return H, Hd, R


@pytest.mark.parametrize("steps", [1, 2, 3])
@pytest.mark.parametrize("bp,dense", [(12, True), (32, False), (256, False)])
def test_precond_fom_breakdown_matches_oracle(bp, dense, steps):
    """The FOM breakdown path of eq. 11's Krylov solve (Sections 3.2, 4.3) on the GPU: dense
    blocks (FOM in each block's FP32 eigenbasis) and the diagonal 256 x 256 tiles (Lanczos on the
    sparse tile in FP32). The even blocks give column 0 an exactly singular 2 x 2 projected
    matrix and the odd blocks give column 1 r^T A r = 0, so the FP32 pivots are rounding noise,
    far below the 1e-4 threshold, and both sides must take the minimal-residual fallback. The
    oracle's results there are pinned to closed forms on the CPU. The random columns 2-3 take a
    shift below every block's spectrum (definite systems): with an indefinite shift a random
    right-hand side can put a pivot near the threshold, where FP32 and FP64 may take different
    branches. Error bound: FP32 work on the block, relative to the largest entry of the reference
    column, 8 b u32 kappa (kappa = ||H~|| / min |lambda - mu|), plus an absolute floor for the
    one-step column whose exact iterate is zero: there the FP32 pivot r^T A r carries the block
    eigendecomposition's error c_J b u32 ||A|| ||r||^2 (c_J <= 14, as in
    test_precond_matches_block_solve), so the fallback iterate is at most 16 b u32 kappa ||r||."""
    import paper_1609_01689_gb300 as lob
    mu = 5.0
    H, Hd, R = _breakdown_matrix(bp, 2, mu, dense, 7 * bp + steps)
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals, precond_block=bp)
    muv = np.array([mu, mu, mu - 5.0, mu - 9.0])
    W = M.precond_apply(t(muv), t(R), solve="fom", steps=steps).cpu().numpy()
    bounds = oracle.uniform_bounds(H.n, bp)
    ref = oracle.block_krylov(H, bounds, muv, R, "fom", steps)
    assert np.all(np.isfinite(W))
    u32 = 2.0 ** -24
    for i in range(len(bounds) - 1):
        s = slice(bounds[i], bounds[i + 1])
        lam = np.linalg.eigvalsh(Hd[s, s])
        for j in range(4):
            kappa = np.abs(lam).max() / np.abs(lam - muv[j]).min()
            scale = np.abs(ref[s, j]).max()
            err = np.abs(W[s, j] - ref[s, j]).max()
            floor = 16 * bp * u32 * kappa * np.linalg.norm(R[s, j])
            assert err <= 8 * bp * u32 * kappa * scale + floor, (i, j, err, scale, kappa)


def _scaled(rng, n, p, spread):
    """Normal entries with per-column and per-row-block scales 2^e, e uniform in [-spread, spread]
    (the digit split's scaling groups are columns of 128-row chunks for the Gram and rows for the
    linear combination), plus one all-zero column."""
    X = rng.standard_normal((n, p))
    X *= 2.0 ** rng.integers(-spread, spread + 1, p)[None, :]
    X *= 2.0 ** rng.integers(-spread, spread + 1, (n + 127) // 128).repeat(128)[:n, None]
    X[:, p // 2] = 0.0
    return X


@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (127, 16, 16), (128, 48, 48), (129, 33, 17), (1000, 64, 64),
                                   (100_000, 48, 48), (70_000, 1, 64), (5000, 64, 1)])
@pytest.mark.parametrize("spread", [0, 20])
def test_gram_tensor_cores(n, p, q, spread):
    """The FP64-class Gram on the tensor cores (p, q <= 64; Ozaki et al.'s error-free digit split).
    Bound, from the split: each operand is truncated at 2^-49 of its scaling group's largest entry
    and every digit product is exact, so per term |err| <= 2^-48 max_group|a| |b| + 2^-48 |a|
    max_group|b|, plus double-float sums (~2^-47 per term). Against the oracle, in the form
    |G - G*| <= 2^-44 (|A|^T |B| + colmax-weighted sums), checked against the double-float kernel
    too. Ragged chunks (n = 127, 129), single rows and columns, column and row-block scales
    spanning 2^40, and a zero column."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n + 7 * p + q + spread)
    A = _scaled(rng, n, p, spread)
    B = _scaled(rng, n, q, spread)
    G = lob.gram(t(A), t(B), "tc").cpu().numpy()
    ref = oracle.gram(A, B)
    # group maxima over 128-row chunks, per column
    nc = (n + 127) // 128
    pad = nc * 128 - n
    Am = np.abs(np.vstack([A, np.zeros((pad, p))])).reshape(nc, 128, p).max(axis=1).repeat(128, axis=0)[:n]
    Bm = np.abs(np.vstack([B, np.zeros((pad, q))])).reshape(nc, 128, q).max(axis=1).repeat(128, axis=0)[:n]
    bound = 2.0 ** -44 * (np.abs(A).T @ np.abs(B) + Am.T @ np.abs(B) + np.abs(A).T @ Bm)
    assert np.all(np.abs(G - ref) <= bound), np.max(np.abs(G - ref) / np.maximum(bound, 1e-300))
    Gd = lob.gram(t(A), t(B), "df64").cpu().numpy()
    assert np.all(np.abs(G - Gd) <= 2 * bound)


@pytest.mark.parametrize("n,p,q", [(1, 1, 1), (127, 48, 16), (4097, 48, 48), (1000, 64, 64), (300, 17, 3)])
@pytest.mark.parametrize("spread", [0, 20])
def test_lincomb_tensor_cores(n, p, q, spread):
    """Y = A C on the tensor cores; scaling groups are the rows of A and the columns of C, so the
    bound carries 2^-44 (|A| |C| + rowmax|A| |C| + |A| colmax|C|)."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n + p + 11 * q + spread)
    A = rng.standard_normal((n, p)) * 2.0 ** rng.integers(-spread, spread + 1, n)[:, None]
    C = rng.standard_normal((p, q)) * 2.0 ** rng.integers(-spread, spread + 1, q)[None, :]
    if p > 2:
        A[:, 1] = 0.0
    Y = lob.lincomb(t(A), t(C), "tc").cpu().numpy()
    ref = oracle.lincomb(A, C)
    ra = np.abs(A).max(axis=1, keepdims=True)
    cc = np.abs(C).max(axis=0, keepdims=True)
    bound = 2.0 ** -44 * (np.abs(A) @ np.abs(C) + ra * np.abs(C).sum(axis=0, keepdims=True) + np.abs(A).sum(
        axis=1, keepdims=True) * cc)
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / np.maximum(bound, 1e-300))
