"""The variable-size block layout that tests/test_gpu_vblock.py holds the GPU store to, pinned on the
CPU: with one group and beta = 256 the blocks are the fixed 256 x 256 tiles, so the layout must
coincide with the oracle's tile builder (orc_tiles) -- same tiles, entries and values, the offsets
repacked from (r << 16) | c into (r << 8) | c -- and for any groups it must list every entry once,
inside blocks that never cross a group start."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_vblock import expected_store


def test_one_group_of_256_rows_is_the_fixed_tile_store():
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    T = oracle.tiles(oracle.Coo(L.n, r, c, v))
    E = expected_store(L.n, r, c, v, [0], 256)
    assert np.array_equal(E["bounds"], np.r_[np.arange(0, L.n, 256), L.n])
    assert np.array_equal(E["tile_rowptr"], T["tile_rowptr"])
    assert np.array_equal(E["tile_col"], T["tile_col"])
    assert np.array_equal(E["tile_ptr"], T["tile_ptr"])
    assert np.array_equal(E["rc16"], (((T["rc"] >> 16) << 8) | (T["rc"] & 0xFFFF)).astype(np.uint16))
    assert np.array_equal(E["v32"], T["v32"])


@pytest.mark.parametrize("beta", [256, 64, 37, 1])
def test_level_aligned_blocks_cover_every_entry_once(beta):
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    groups = synth.level_starts(L)[:-1]
    E = expected_store(L.n, r, c, v, groups, beta)
    b = E["bounds"]
    assert b[0] == 0 and b[-1] == L.n and (np.diff(b) >= 1).all() and (np.diff(b) <= beta).all()
    # no block crosses a group start
    for g in groups:
        assert g in b
    # every entry once: rebuild (row, col) from the blocks
    nt = len(E["tile_col"])
    tr = np.repeat(np.searchsorted(E["tile_rowptr"], np.arange(nt), side="right") - 1, np.diff(E["tile_ptr"]))
    tc = np.repeat(E["tile_col"], np.diff(E["tile_ptr"]))
    rows = b[tr] + (E["rc16"] >> 8)
    cols = b[tc] + (E["rc16"] & 0xFF)
    assert np.array_equal(np.sort(rows * L.n + cols), np.sort(r * L.n + c))
    # entries of a block in (r, c) order, blocks in (block row, block column) order
    nblk = len(b) - 1
    key = (tr.astype(np.int64) * nblk + tc) * 65536 + E["rc16"]
    assert (np.diff(key) > 0).all()
