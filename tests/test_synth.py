"""The seeded input generator: level layout, structure and value statistics, determinism."""
import numpy as np
import pytest

import synth
from conftest import golden_path


def test_level_counts_c1_golden():
    expect = [int(x) for x in open(golden_path("levels_c1.txt")).read().split("\n")[-2].split()]
    L = synth.config_layout("c1")
    assert np.diff(synth.level_starts(L)).tolist() == expect


@pytest.mark.parametrize("n,Q", [(1, 0), (10, 3), (1536, 6), (500_000, 10), (8_000_000, 14)])
def test_level_counts_sum_and_grow(n, Q):
    L = synth.layout(n, Q, 30, 1)
    c = np.diff(synth.level_starts(L))
    assert c.sum() == n and len(c) == Q + 1
    big = c[:-1] >= 100  # rounding dominates the ratio of small levels
    ratio = c[1:][big] / c[:-1][big]
    assert np.all(np.abs(ratio - 2.2) < 0.02)


@pytest.fixture(scope="module")
def c1():
    L = synth.config_layout("c1")
    return L, synth.generate(L)


def test_structure(c1):
    L, (r, c, v) = c1
    n = L.n
    assert np.all(r <= c)
    key = r * n + c
    assert np.all(np.diff(key) > 0)  # sorted, unique
    assert np.array_equal(r[r == c], np.arange(n))  # full diagonal
    lev = np.searchsorted(synth.level_starts(L), np.arange(n), side="right") - 1
    assert np.all(np.abs(lev[r] - lev[c]) <= 2)  # coupling only between nearby levels
    full_per_row = (2 * len(r) - n) / n
    assert abs(full_per_row - 30) <= 4


def test_value_statistics(c1):
    L, (r, c, v) = c1
    off = v[r != c]
    m = len(off)
    assert abs(off.mean()) <= 4 * 0.3 / np.sqrt(m)
    assert abs(off.var() - 0.09) <= 0.09 * 6 * np.sqrt(2.0 / m)
    assert np.abs(off).max() <= 0.3 * 6
    lev = np.searchsorted(synth.level_starts(L), np.arange(L.n), side="right") - 1
    d = v[r == c]
    assert np.all(np.abs(d - 10 * lev) <= 1.0)


def test_deterministic_and_seeded():
    L1 = synth.layout(3000, 7, 40, 5)
    a = synth.generate(L1)
    b = synth.generate(synth.layout(3000, 7, 40, 5))
    c = synth.generate(synth.layout(3000, 7, 40, 6))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not (len(a[0]) == len(c[0]) and np.array_equal(a[2], c[2]))


def test_interp_levels():
    assert synth.interp_levels(1536) == 6
    assert synth.interp_levels(500_000) == 10
    assert synth.interp_levels(8_000_000) == 14
    assert synth.interp_levels(100) == 6 and synth.interp_levels(10**9) == 14
