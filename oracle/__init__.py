"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct FP64 CPU reference (``oracle.c``) for what the GPU path
computes, wrapped with ctypes. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it. It shares no code with the CUDA library.

Functions follow the paper as cited in ``oracle.c``: the k smallest eigenpairs of a
symmetric H stored as one triangle (Section 3.1, eq. 6), by dense Householder+QL, by cyclic
Jacobi and by Lanczos with full reorthogonalisation; plus the pieces of one LOBPCG
iteration with their plain definitions (symmetric SpMM, Section 4.1; block inner products
and linear combinations, Section 4.4; block-diagonal preconditioner, eq. 11;
Rayleigh-Ritz, eq. 9) and the CSB tile store (Sections 2.2 and 4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

_P = ctypes.c_void_p
_I = ctypes.c_int64
_D = ctypes.c_double


def build() -> str:
    if not os.path.exists(_SO) or os.path.getmtime(_SRC) > os.path.getmtime(_SO):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", _SO, _SRC,
                               "-lm"])
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_spmm.argtypes = [_I, _I, _P, _P, _P, _I, _P, _P]
        L.orc_spmm_csr.argtypes = [_I, _P, _P, _P, _I, _P, _P]
        L.orc_lanczos_csr.argtypes = [_I, _P, _P, _P, _I, _D, _D, _I, ctypes.c_uint64, _P, _P, _P]
        L.orc_lanczos_csr.restype = ctypes.c_int
        L.orc_dense.argtypes = [_I, _I, _P, _P, _P, _P]
        L.orc_norm_inf.argtypes = [_I, _I, _P, _P, _P]
        L.orc_norm_inf.restype = _D
        L.orc_tridiag_eig.argtypes = [_I, _P, _P, _P, _I, _I]
        L.orc_tridiag_eig.restype = ctypes.c_int
        L.orc_syev.argtypes = [_I, _P, _P]
        L.orc_syev.restype = ctypes.c_int
        L.orc_jacobi.argtypes = [_I, _P, _P, _P, ctypes.c_int]
        L.orc_jacobi.restype = ctypes.c_int
        L.orc_lanczos.argtypes = [_I, _I, _P, _P, _P, _I, _D, _D, _I, ctypes.c_uint64, _P, _P, _P]
        L.orc_lanczos.restype = ctypes.c_int
        L.orc_tiles.argtypes = [_I, _I, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P]
        L.orc_tiles.restype = _I
        L.orc_gram.argtypes = [_I, _I, _P, _I, _P, _P]
        L.orc_lincomb.argtypes = [_I, _I, _P, _I, _P, _P]
        L.orc_block_precond.argtypes = [_I, _I, _P, _P, _P, _I, _P, _I, _P, _P, _P]
        L.orc_block_krylov.argtypes = [_I, _I, _P, _P, _P, _I, _P, _I, _P, _P, ctypes.c_int, ctypes.c_int, _D, _P]
        L.orc_block_precond.restype = ctypes.c_int
        L.orc_rayleigh_ritz.argtypes = [_I, _P, _P, _P, _P]
        L.orc_rayleigh_ritz.restype = ctypes.c_int
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


class Coo:
    """Upper triangle (row <= col) incl. diagonal of a symmetric n x n matrix."""

    def __init__(self, n, rows, cols, vals):
        self.n = int(n)
        self.rows = _i64(rows)
        self.cols = _i64(cols)
        self.vals = _f64(vals)
        self.nnz = len(self.rows)

    def args(self):
        return (self.n, self.nnz, self.rows.ctypes.data, self.cols.ctypes.data, self.vals.ctypes.data)


def spmm(H: Coo, X: np.ndarray) -> np.ndarray:
    """Y = H X (Section 4.1: each stored h_ij applied as h_ij and h_ji)."""
    X = _f64(X)
    nb = 1 if X.ndim == 1 else X.shape[1]
    Y = np.empty_like(X)
    lib().orc_spmm(*H.args(), nb, X.ctypes.data, Y.ctypes.data)
    return Y


def dense(H: Coo) -> np.ndarray:
    A = np.empty((H.n, H.n), dtype=np.float64)
    lib().orc_dense(*H.args(), A.ctypes.data)
    return A


def norm_inf(H: Coo) -> float:
    return float(lib().orc_norm_inf(*H.args()))


def syev(A: np.ndarray):
    """All eigenpairs of dense symmetric A by Householder tridiagonalisation + implicit QL."""
    A = _f64(A).copy()
    n = A.shape[0]
    w = np.empty(n, dtype=np.float64)
    if lib().orc_syev(n, A.ctypes.data, w.ctypes.data) != 0:
        raise RuntimeError("QL did not converge")
    return w, A


def tridiag_eig(d, e):
    d = _f64(d).copy()
    e = _f64(e)
    m = len(d)
    Z = np.eye(m, dtype=np.float64)
    if lib().orc_tridiag_eig(m, d.ctypes.data, e.ctypes.data, Z.ctypes.data, m, m) != 0:
        raise RuntimeError("QL did not converge")
    return d, Z


def jacobi(A: np.ndarray, max_sweeps: int = 100):
    """All eigenpairs of dense symmetric A by cyclic Jacobi rotations."""
    A = _f64(A).copy()
    n = A.shape[0]
    w = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.float64)
    sw = lib().orc_jacobi(n, A.ctypes.data, w.ctypes.data, V.ctypes.data, max_sweeps)
    if sw < 0:
        raise RuntimeError("Jacobi did not converge")
    return w, V


def lanczos(H: Coo, k: int, tol: float, normH: float | None = None, max_steps: int = 2000, seed: int = 7):
    """k smallest Ritz pairs by Lanczos with full reorthogonalisation; stops when the Ritz
    residual estimates are <= tol * ||H||. Returns (lam, X, steps, converged)."""
    if normH is None:
        normH = norm_inf(H)
    lam = np.zeros(k, dtype=np.float64)
    X = np.zeros((H.n, k), dtype=np.float64)
    steps = ctypes.c_int64(0)
    st = lib().orc_lanczos(*H.args(), k, tol, normH, max_steps, seed, lam.ctypes.data, X.ctypes.data,
                           ctypes.byref(steps))
    if st < 0:
        raise RuntimeError(f"Lanczos failed ({st})")
    return lam, X, int(steps.value), st == 0


class Csr:
    """Upper triangle (row <= col) incl. diagonal in CSR form: rowptr (n+1, int64), col (int32),
    val (float64), rows in order and columns in order within each row."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = _i64(rowptr)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)
        assert self.rowptr.shape == (self.n + 1,) and len(self.col) == len(self.val) == int(self.rowptr[-1])

    @staticmethod
    def from_sorted_coo(n, rows, cols, vals):
        """From a COO sorted by (row, col) (the generator's order)."""
        rowptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
        return Csr(n, rowptr, cols.astype(np.int32), vals)

    def args(self):
        return (self.n, self.rowptr.ctypes.data, self.col.ctypes.data, self.val.ctypes.data)


def spmm_csr(H: Csr, X: np.ndarray) -> np.ndarray:
    """spmm on the CSR form (orc_spmm_csr)."""
    X = _f64(X)
    nb = 1 if X.ndim == 1 else X.shape[1]
    Y = np.empty_like(X)
    lib().orc_spmm_csr(*H.args(), nb, X.ctypes.data, Y.ctypes.data)
    return Y


def lanczos_csr(H: Csr, k: int, tol: float, normH: float, max_steps: int = 2000, seed: int = 7):
    """lanczos on the CSR form (orc_lanczos_csr). Returns (lam, X, steps, converged)."""
    lam = np.zeros(k, dtype=np.float64)
    X = np.zeros((H.n, k), dtype=np.float64)
    steps = ctypes.c_int64(0)
    st = lib().orc_lanczos_csr(*H.args(), k, tol, normH, max_steps, seed, lam.ctypes.data, X.ctypes.data,
                               ctypes.byref(steps))
    if st < 0:
        raise RuntimeError(f"Lanczos failed ({st})")
    return lam, X, int(steps.value), st == 0


def eigh_small(H: Coo, k: int):
    """k smallest eigenpairs of a small sparse H via the dense solver."""
    w, Z = syev(dense(H))
    return w[:k], Z[:, :k]


def tiles(H: Coo, b: int = 256):
    """CSB tile store of H (see orc_tiles): dict of numpy arrays, bit-exact reference."""
    nt = (H.n + b - 1) // b
    rowptr = np.empty(nt + 1, dtype=np.int64)
    tcol = np.empty(max(H.nnz, 1), dtype=np.int32)
    tptr = np.empty(max(H.nnz, 1) + 1, dtype=np.int64)
    rc = np.empty(max(H.nnz, 1), dtype=np.uint32)
    v64 = np.empty(max(H.nnz, 1), dtype=np.float64)
    v32 = np.empty(max(H.nnz, 1), dtype=np.float32)
    ntiles = lib().orc_tiles(*H.args(), b, rowptr.ctypes.data, tcol.ctypes.data, tptr.ctypes.data, rc.ctypes.data,
                             v64.ctypes.data, v32.ctypes.data)
    if ntiles < 0:
        raise ValueError({-1: "entry out of range", -2: "entry below the diagonal", -3: "duplicate entry",
                          -4: "bad tile size"}[ntiles])
    return dict(tile_rowptr=rowptr, tile_col=tcol[:ntiles].copy(), tile_ptr=tptr[:ntiles + 1].copy(),
                rc=rc[:H.nnz].copy(), v64=v64[:H.nnz].copy(), v32=v32[:H.nnz].copy(), ntiles=int(ntiles))


def gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A^T B for tall-skinny row-major blocks (Section 4.4)."""
    A = _f64(A); B = _f64(B)
    G = np.empty((A.shape[1], B.shape[1]), dtype=np.float64)
    lib().orc_gram(A.shape[0], A.shape[1], A.ctypes.data, B.shape[1], B.ctypes.data, G.ctypes.data)
    return G


def lincomb(A: np.ndarray, C: np.ndarray) -> np.ndarray:
    """A C for a tall-skinny A (Section 4.4, eq. 7)."""
    A = _f64(A); C = _f64(C)
    Y = np.empty((A.shape[0], C.shape[1]), dtype=np.float64)
    lib().orc_lincomb(A.shape[0], A.shape[1], A.ctypes.data, C.shape[1], C.ctypes.data, Y.ctypes.data)
    return Y


def block_precond(H: Coo, bounds, mu, R: np.ndarray) -> np.ndarray:
    """W with (H~_[i] - mu_j I) W_[i] = R_[i] for the diagonal blocks given by bounds (eq. 11)."""
    bounds = _i64(bounds)
    mu = _f64(mu)
    R = _f64(R)
    W = np.empty_like(R)
    st = lib().orc_block_precond(*H.args(), len(bounds) - 1, bounds.ctypes.data, R.shape[1], mu.ctypes.data,
                                 R.ctypes.data, W.ctypes.data)
    if st != 0:
        raise ZeroDivisionError("singular block system")
    return W


KRYLOV = {"fom": 0, "minres": 2, "abs": 3}


def block_krylov(H: Coo, bounds, mu, R: np.ndarray, method: str, steps: int = 3, guard: float = 0.0) -> np.ndarray:
    """Approximate eq. 11 solves per block and column: FOM or minimal residual with `steps`
    Krylov iterations from a zero start, or |H~_[i] - mu_j I|^{-1} ('abs')."""
    bounds = _i64(bounds)
    assert np.diff(bounds).max() <= 256
    mu = _f64(mu)
    R = _f64(R)
    W = np.empty_like(R)
    st = lib().orc_block_krylov(*H.args(), len(bounds) - 1, bounds.ctypes.data, R.shape[1], mu.ctypes.data,
                                R.ctypes.data, KRYLOV[method], steps, guard, W.ctypes.data)
    if st != 0:
        raise RuntimeError("block eigendecomposition failed")
    return W


def uniform_bounds(n: int, bp: int) -> np.ndarray:
    return np.array(list(range(0, n, bp)) + [n], dtype=np.int64)


def rayleigh_ritz(G: np.ndarray, M: np.ndarray):
    """theta, C with G C = M C diag(theta), C^T M C = I (eq. 9)."""
    G = _f64(G); M = _f64(M)
    m = G.shape[0]
    theta = np.empty(m, dtype=np.float64)
    C = np.empty((m, m), dtype=np.float64)
    st = lib().orc_rayleigh_ritz(m, G.ctypes.data, M.ctypes.data, theta.ctypes.data, C.ctypes.data)
    if st == -1:
        raise np.linalg.LinAlgError("Gram matrix not positive definite")
    if st != 0:
        raise RuntimeError("QL did not converge")
    return theta, C


def residual_norms(H: Coo, X: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """||H x_j - lam_j x_j|| for each column (Algorithm 1, step 4)."""
    R = spmm(H, X) - X * lam[None, :]
    return np.sqrt((R * R).sum(axis=0))
