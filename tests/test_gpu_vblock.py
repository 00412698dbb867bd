"""Variable-size CSB blocks with 8 + 8-bit offsets (Section 2.2, Section 4.2; lob_v*).

The store must equal, array by array and bit for bit, the layout written out here from its
definition: blocks cut from the caller's groups (at most beta_max rows each, starting at each
group's start), nonzero blocks in (block row, block column) order, entries inside a block in
(r, c) order as (r << 8) | c with the value rounded to FP32; and it must round-trip to the input
COO. The product is checked like the fixed-tile one: integer data exactly, random data within
2 (m + 4) u32 (|H||X|) per entry (X and values rounded to FP32, FP32 products and in-block sums)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import abs_coo, random_upper, row_counts

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def expected_store(n, rows, cols, vals, groups, beta):
    bnd = []
    ext = list(groups) + [n]
    for i in range(len(groups)):
        bnd += list(range(ext[i], ext[i + 1], beta))
    bnd = np.array(bnd + [n], np.int64)
    bi = np.searchsorted(bnd, rows, side="right") - 1
    bj = np.searchsorted(bnd, cols, side="right") - 1
    r = rows - bnd[bi]
    c = cols - bnd[bj]
    order = np.lexsort((c, r, bj, bi))
    bi, bj, r, c, v = bi[order], bj[order], r[order], c[order], vals[order]
    new = np.r_[True, (bi[1:] != bi[:-1]) | (bj[1:] != bj[:-1])]
    starts = np.nonzero(new)[0]
    tile_row = bi[starts]
    nblk = len(bnd) - 1
    return dict(bounds=bnd, tile_rowptr=np.searchsorted(tile_row, np.arange(nblk + 1), side="left").astype(np.int64),
                tile_col=bj[starts].astype(np.int32), tile_ptr=np.r_[starts, len(order)].astype(np.int64),
                rc16=((r << 8) | c).astype(np.uint16), v32=v.astype(np.float32))


@pytest.mark.parametrize("beta", [256, 64, 37])
def test_vblock_store_matches_its_definition_and_round_trips(beta):
    import paper_1609_01689_gb300 as lob
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    groups = synth.level_starts(L)[:-1]
    perm = np.random.default_rng(beta).permutation(len(r))
    V = lob.VMatrix(L.n, r[perm], c[perm], v[perm], groups, beta)
    got = V.export()
    exp = expected_store(L.n, r, c, v, groups, beta)
    for key in exp:
        assert np.array_equal(got[key], exp[key]), key
    info = V.info()
    assert info["nnz"] == len(r) and info["nblocks"] == len(exp["bounds"]) - 1
    assert info["store_bytes"] < 8 * len(r) + 16 * (info["nblocks"] + 1) + 12 * info["ntiles"]
    # every block lies inside one group and has at most beta rows
    b = got["bounds"]
    assert (np.diff(b) <= beta).all() and set(groups.tolist()) <= set(b.tolist())
    # round trip: global (row, col) and the FP32 values
    nt = len(got["tile_col"])
    tr = np.repeat(np.searchsorted(got["tile_rowptr"], np.arange(nt), side="right") - 1, np.diff(got["tile_ptr"]))
    tc = np.repeat(got["tile_col"], np.diff(got["tile_ptr"]))
    rows = b[tr] + (got["rc16"] >> 8)
    cols = b[tc] + (got["rc16"] & 0xFF)
    key_in = np.lexsort((c, r))
    key_out = np.lexsort((cols, rows))
    assert np.array_equal(rows[key_out], r[key_in]) and np.array_equal(cols[key_out], c[key_in])
    assert np.array_equal(got["v32"][key_out], v[key_in].astype(np.float32))
    V.close()


def test_vblock_rejects_bad_groups():
    import paper_1609_01689_gb300 as lob
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    for groups, beta in (([1, 5], 64), ([0, 10, 10], 64), ([0, L.n], 64), ([0], 0), ([0], 257)):
        with pytest.raises(lob.LobError):
            lob.VMatrix(L.n, r, c, v, groups, beta)


@pytest.mark.parametrize("nb", [1, 7, 16])
def test_vblock_spmm_integer_exact(nb):
    import torch

    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(nb)
    H = random_upper(1300, 0.06, rng, integer=True)
    X = rng.integers(-8, 9, (1300, nb)).astype(np.float64)
    V = lob.VMatrix(H.n, H.rows, H.cols, H.vals, [0, 100, 333, 900], 200)
    Y = V.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(Y, oracle.spmm(H, X))


def test_vblock_spmm_dense_blocks_span_chunks():
    """Dense blocks hold several 4,096-entry chunks of the permutation."""
    import torch

    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(5)
    H = random_upper(700, 0.8, rng, integer=True)
    X = rng.integers(-4, 5, (700, 16)).astype(np.float64)
    V = lob.VMatrix(H.n, H.rows, H.cols, H.vals, [0, 300], 256)
    assert np.array_equal(V.spmm(torch.from_numpy(X).cuda()).cpu().numpy(), oracle.spmm(H, X))


def test_vblock_spmm_within_bound_on_the_level_structure():
    import torch

    import paper_1609_01689_gb300 as lob
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    X = np.random.default_rng(3).standard_normal((L.n, 16))
    V = lob.VMatrix(L.n, r, c, v, synth.level_starts(L)[:-1], 128)
    Y = V.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    bound = 2 * (row_counts(H)[:, None] + 4) * U32 * oracle.spmm(abs_coo(H), np.abs(X))
    assert np.all(np.abs(Y - oracle.spmm(H, X)) <= bound)


def test_vblock_spmm_full_size_500k_matches_fixed_tiles():
    """The n = 500,000 workload with level-aligned 256-row blocks: the same product as the fixed-tile
    FP32-value kernel within the sum of both bounds, on sampled rows checked against the oracle."""
    import torch

    import paper_1609_01689_gb300 as lob
    L = synth.config_layout("c2")
    r, c, v = synth.generate_device(L)
    V = lob.VMatrix(L.n, r, c, v, synth.level_starts(L)[:-1], 256)
    M = lob.Matrix(L.n, r, c, v)
    X = torch.randn((L.n, 16), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(9))
    Yv = V.spmm(X)
    Yf = M.spmm(X, "mixed")
    H = oracle.Coo(L.n, r.cpu().numpy(), c.cpu().numpy(), v.cpu().numpy())
    Xh = X.cpu().numpy()
    bound = 2 * (row_counts(H)[:, None] + 4) * U32 * oracle.spmm(abs_coo(H), np.abs(Xh))
    Yref = oracle.spmm(H, Xh)
    assert np.all(np.abs(Yv.cpu().numpy() - Yref) <= bound)
    assert np.all(np.abs(Yv.cpu().numpy() - Yf.cpu().numpy()) <= 2 * bound)
    V.close()
    M.close()
