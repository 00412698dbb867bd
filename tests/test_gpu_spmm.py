"""Symmetric SpMM Y = H X (Section 4.1) against the oracle, in FP64 and in the mixed
arithmetic (FP32 values and products, FP64 sums across tiles; footnote 5 of Section 4.4).

Bounds: FP64 -- |Y - Y*| <= 2 (m + 2) u64 (|H||X|) per entry, m = nonzeros in the row.
        MIXED -- X and values rounded to FP32 (2 u32 each), FP32 products and in-tile sums
        (m u32): |Y - Y*| <= 2 (m + 4) u32 (|H||X|)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import abs_coo, random_upper, row_counts

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def run(M, X, mode):
    import torch
    return M.spmm(torch.from_numpy(np.ascontiguousarray(X)).cuda(), mode).cpu().numpy()


@pytest.mark.parametrize("nb", [1, 3, 8, 16, 17, 64])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_spmm_integer_exact(nb, mode):
    """Small integers: every product and partial sum is exact in both arithmetics."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(nb + 100 * (mode == "mixed"))
    H = random_upper(700, 0.05, rng, integer=True)
    X = rng.integers(-8, 9, (700, nb)).astype(np.float64)
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    assert np.array_equal(run(M, X, mode), oracle.spmm(H, X))


@pytest.mark.parametrize("n,density,nb", [(600, 0.9, 16), (520, 0.45, 17), (1100, 0.12, 16)])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "df64"])
def test_spmm_dense_tiles_integer_exact(n, density, nb, mode):
    """Dense tiles: a tile spans several chunks of the column permutation, so the ring kernels'
    stages hold consecutive chunks of one tile and X_J is staged once per chunk."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n + nb)
    H = random_upper(n, density, rng, integer=True)
    X = rng.integers(-4, 5, (n, nb)).astype(np.float64)
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    assert np.array_equal(run(M, X, mode), oracle.spmm(H, X))


@pytest.mark.parametrize("n,nb", [(1, 1), (1, 16), (200, 16), (255, 4), (256, 8), (257, 16), (3000, 16), (5000, 2)])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "df64"])
def test_spmm_random_within_bound(n, nb, mode):
    """Random data within the rounding bound of each arithmetic, from one entry to several tile rows (nb = 16 runs
    the ring kernels with one persistent CTA per tile-row range)."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n * 7 + nb)
    H = random_upper(n, min(0.05, 40.0 / n), rng)
    X = rng.standard_normal((n, nb))
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    Y = run(M, X, mode)
    Yref = oracle.spmm(H, X)
    bound_base = oracle.spmm(abs_coo(H), np.abs(X))
    m = row_counts(H)[:, None]
    unit = {"fp64": 2 * (m + 2) * U64, "mixed": 2 * (m + 4) * U32, "df64": 2 * (m + 2) * 2.0 ** -46}[mode]
    assert np.all(np.abs(Y - Yref) <= unit * bound_base + 1e-300)


def test_spmm_unit_vectors_and_symmetry():
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(5)
    H = random_upper(600, 0.03, rng)
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    cols = [0, 255, 256, 599]
    E = np.zeros((600, len(cols)))
    E[cols, range(len(cols))] = 1.0
    A = oracle.dense(H)
    assert np.array_equal(run(M, E, "fp64"), A[:, cols])
    X = rng.standard_normal((600, 4)); Z = rng.standard_normal((600, 4))
    lhs = X.T @ run(M, Z, "fp64"); rhs = run(M, X, "fp64").T @ Z
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


def test_spmm_diagonal_only_and_single_entry():
    import paper_1609_01689_gb300 as lob
    d = np.arange(1.0, 301.0)
    M = lob.Matrix(300, np.arange(300), np.arange(300), d)
    X = np.ones((300, 2))
    assert np.array_equal(run(M, X, "fp64"), d[:, None] * X)
    M1 = lob.Matrix(600, np.array([10]), np.array([590]), np.array([2.5]))
    Y = run(M1, np.ones((600, 1)), "fp64")
    expect = np.zeros((600, 1)); expect[10] = 2.5; expect[590] = 2.5
    assert np.array_equal(Y, expect)


@pytest.fixture(scope="module")
def c2():
    L = synth.config_layout("c2")
    r, c, v = synth.generate(L)
    return L, oracle.Coo(L.n, r, c, v)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "df64"])
def test_spmm_full_size_500k(c2, mode):
    """The n = 500,000, nb = 16 workload in the launch configuration the benchmark times (the ring
    kernels for the FP32-value and double-float products)."""
    import paper_1609_01689_gb300 as lob
    L, H = c2
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    rng = np.random.default_rng(16)
    X = rng.standard_normal((H.n, 16))
    Y = run(M, X, mode)
    Yref = oracle.spmm(H, X)
    bound_base = oracle.spmm(abs_coo(H), np.abs(X))
    m = row_counts(H)[:, None]
    unit = {"fp64": 2 * (m + 2) * U64, "mixed": 2 * (m + 4) * U32, "df64": 2 * (m + 2) * 2.0 ** -46}[mode]
    assert np.all(np.abs(Y - Yref) <= unit * bound_base)


@pytest.mark.parametrize("nb", [1, 2, 5, 8, 16, 24])
def test_spmm_df64_integer_exact_and_fp64_class(nb):
    """FP64-class double-float products (LOB_SPMM_DF64): exact on small integers; on random data
    within the FP64 bound with a double-float unit: |Y - Y*| <= 2 (m + 2) 2^-46 (|H||X|)."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(300 + nb)
    H = random_upper(900, 0.04, rng, integer=True)
    X = rng.integers(-8, 9, (900, nb)).astype(np.float64)
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    assert np.array_equal(run(M, X, "df64"), oracle.spmm(H, X))
    H = random_upper(900, 0.04, rng)
    X = rng.standard_normal((900, nb))
    M = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    Y = run(M, X, "df64")
    bound = 2 * (row_counts(H)[:, None] + 2) * 2.0 ** -46 * oracle.spmm(abs_coo(H), np.abs(X))
    assert np.all(np.abs(Y - oracle.spmm(H, X)) <= bound)


@pytest.mark.parametrize("mode", ["mixed", "df64"])
def test_spmm_bounded_wait_reports_and_context_survives(mode):
    """Failure detection without a GPU fault: a matrix created in the wait test mode
    (wait_log2 = -1) makes the first pipeline stage of the persistent SpMM kernels (nb = 16) wait
    for bytes that nothing sends, so that wait runs out every time. The kernel must then stop
    issuing copies, let the copies already in flight land, leave, and set the matrix's status word: lob_check reports LOB_ERR_CUDA once (then the word is clear), a
    solve on that matrix returns LOB_ERR_CUDA, and a product on a normally created matrix right
    after is exact (the context stays usable)."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(77)
    H = random_upper(3000, 0.01, rng, integer=True)
    X = rng.integers(-8, 9, (3000, 16)).astype(np.float64)
    Mbad = lob.Matrix(H.n, H.rows, H.cols, H.vals, wait_log2=-1)
    run(Mbad, X, mode)
    with pytest.raises(lob.LobError) as e:
        Mbad.check()
    assert e.value.code == lob.LOB_ERR_CUDA
    Mbad.check()  # cleared
    if mode == "mixed":
        with pytest.raises(lob.LobError) as e:
            Mbad.solve(4, 16, 1e-8, mode="mixed", max_iter=5)
        assert e.value.code == lob.LOB_ERR_CUDA
    Mok = lob.Matrix(H.n, H.rows, H.cols, H.vals)
    assert np.array_equal(run(Mok, X, mode), oracle.spmm(H, X))
    Mok.check()
