"""Helpers shared by the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np

import oracle


def random_upper(n, density, rng, integer=False, lo=-8, hi=8):
    """Upper triangle incl. a full diagonal of a random symmetric n x n matrix (COO)."""
    if n <= 3000:
        mask = np.triu(rng.random((n, n)) < density, 1) | np.eye(n, dtype=bool)
        r, c = np.nonzero(mask)
    else:
        m = int(density * n * n / 2)
        a = rng.integers(0, n, m); b = rng.integers(0, n, m)
        r0, c0 = np.minimum(a, b), np.maximum(a, b)
        key = np.unique(np.concatenate([r0 * n + c0, np.arange(n) * (n + 1)]))
        r, c = key // n, key % n
    if integer:
        v = rng.integers(lo, hi + 1, len(r)).astype(np.float64)
    else:
        v = rng.standard_normal(len(r))
    return oracle.Coo(n, r.astype(np.int64), c.astype(np.int64), v)


def abs_coo(H):
    return oracle.Coo(H.n, H.rows, H.cols, np.abs(H.vals))


def row_counts(H):
    cnt = np.bincount(H.rows, minlength=H.n) + np.bincount(H.cols[H.rows != H.cols], minlength=H.n)
    return cnt
