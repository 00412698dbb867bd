"""Tile-store build on the GPU (Sections 2.2 and 4.2) is bit-exact against the oracle's CPU
builder, for ragged, tiny and generated matrices, from host and device COO."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import random_upper

pytestmark = pytest.mark.gpu


def compare(M, H):
    import paper_1609_01689_gb300 as lob  # noqa: F401
    got = M.export_tiles()
    ref = oracle.tiles(H, 256)
    assert got["ntiles"] == ref["ntiles"]
    for key in ("tile_rowptr", "tile_col", "tile_ptr", "rc", "v64", "v32"):
        a, b = got[key], ref[key]
        assert a.dtype == b.dtype and a.shape == b.shape, key
        assert a.tobytes() == b.tobytes(), key


CASES = [("single", 1), ("tiny", 5), ("ragged", 300), ("two_tiles", 513), ("mid", 2000)]


@pytest.mark.parametrize("name,n", CASES)
def test_tiles_bit_exact_random(name, n):
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n)
    H = random_upper(n, 0.05, rng)
    perm = rng.permutation(H.nnz)
    M = lob.Matrix(n, H.rows[perm], H.cols[perm], H.vals[perm])
    compare(M, H)


def test_tiles_bit_exact_generated_c1_and_100k():
    import paper_1609_01689_gb300 as lob
    for L in (synth.config_layout("c1"), synth.layout(100_000, 9, 60, 3)):
        r, c, v = synth.generate(L)
        H = oracle.Coo(L.n, r, c, v)
        compare(lob.Matrix(L.n, r, c, v), H)


def test_tiles_from_device_coo_and_device_generator():
    import torch
    import paper_1609_01689_gb300 as lob
    L = synth.layout(20_000, 8, 40, 9)
    r, c, v = synth.generate(L)
    dr, dc, dv = synth.generate_device(L)
    assert np.array_equal(dr.cpu().numpy(), r) and np.array_equal(dc.cpu().numpy(), c)
    assert dv.cpu().numpy().tobytes() == v.tobytes()  # host and device generators agree bit for bit
    perm = torch.randperm(len(r), device="cuda")
    M = lob.Matrix(L.n, dr[perm], dc[perm], dv[perm])
    compare(M, oracle.Coo(L.n, r, c, v))


def test_tiles_reject_bad_entries():
    import paper_1609_01689_gb300 as lob
    with pytest.raises(lob.LobError) as e:
        lob.Matrix(4, np.array([0, 0]), np.array([1, 1]), np.array([1.0, 1.0]))  # duplicate
    assert e.value.code == lob.LOB_ERR_ARG
    with pytest.raises(lob.LobError):
        lob.Matrix(4, np.array([2]), np.array([1]), np.array([1.0]))  # below the diagonal
    with pytest.raises(lob.LobError):
        lob.Matrix(4, np.array([0]), np.array([4]), np.array([1.0]))  # out of range


def expected_perm(T, chunk):
    """Chunk-local (column, row)-order permutation rebuilt from the canonical store."""
    rc = T["rc"].astype(np.int64)
    tp = T["tile_ptr"]
    out = np.empty(len(rc), np.uint16)
    for t in range(T["ntiles"]):
        for b in range(tp[t], tp[t + 1], chunk):
            e = min(b + chunk, tp[t + 1])
            seg = rc[b:e]
            key = (seg & 0xFFFF) * 65536 + (seg >> 16)
            out[b:e] = np.argsort(key, kind="stable").astype(np.uint16)
    return out


@pytest.mark.parametrize("n,density", [(700, 0.05), (3000, 0.4)])
def test_column_permutation_round_trips(n, density):
    """The kernel-private permutation is exactly the (c, r) order of each chunk, including tiles
    longer than one chunk (density 0.4 gives ~13k entries per diagonal-region tile)."""
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(n)
    H = random_upper(n, density, rng)
    M = lob.Matrix(n, H.rows, H.cols, H.vals)
    T = M.export_tiles()
    chunk = M.info()["perm_chunk"]
    assert chunk in (1024, 2048, 4096)
    assert np.array_equal(M.export_perm(), expected_perm(T, chunk))
