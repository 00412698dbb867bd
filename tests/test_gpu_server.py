"""Serving: the batched SpMM launch and the continuous-batching server against the oracle.

Acceptance (as for lob_solve): eigenvalues within 1e-9 (FP64 path) or 1e-8 (mixed path) of the
oracle's in |lambda - lambda*| / max(|lambda*|, 1); residuals <= tol ||H||. A solve in the mix
must agree with the same solve run alone to 1e-10 in that measure (both converge to the same
eigenpairs; only the unordered atomic column sums of the SpMM differ between runs)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import random_upper

pytestmark = pytest.mark.gpu


def test_spmm_batch_integer_exact():
    """Integer-valued H and X: every sum is exact in each arithmetic, so each batched product
    equals the oracle's bit for bit, whatever the neighbours in the launch."""
    import torch
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(7)
    sizes = [300, 1000, 2500, 700, 257, 1]
    widths = [1, 4, 8, 16, 3, 2]
    modes = ["fp64", "mixed", "df64", "mixed", "fp64", "df64"]
    Hs, mats, Xs = [], [], []
    for n, w in zip(sizes, widths):
        H = random_upper(n, min(1.0, 40.0 / n), rng, integer=True)
        Hs.append(H)
        mats.append(lob.Matrix(n, H.rows, H.cols, H.vals))
        Xs.append(rng.integers(-8, 9, (n, w)).astype(np.float64))
    Ys = lob.spmm_batch(mats, Xs, modes)
    torch.cuda.synchronize()
    for H, X, Y in zip(Hs, Xs, Ys):
        np.testing.assert_array_equal(Y.cpu().numpy(), oracle.spmm(H, X))


@pytest.mark.parametrize("mode", ["fp64", "mixed", "df64"])
def test_spmm_batch_leading_block_never_reads_beyond(mode):
    """With n_act the product is the leading block's: rows of X at or beyond n_act are not read
    (NaN there must not reach Y), and rows below n_act equal the oracle product of the leading
    block (integer data: exact in every arithmetic)."""
    import torch
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(11)
    sizes, nacts = [900, 1300, 520], [47, 700, 300]
    Hs, mats, Xs = [], [], []
    for n in sizes:
        H = random_upper(n, 30.0 / n, rng, integer=True)
        Hs.append(H)
        mats.append(lob.Matrix(n, H.rows, H.cols, H.vals))
    for n, na in zip(sizes, nacts):
        X = rng.integers(-8, 9, (n, 4)).astype(np.float64)
        X[na:] = np.nan
        Xs.append(X)
    Ys = lob.spmm_batch(mats, Xs, mode, n_act=nacts)
    torch.cuda.synchronize()
    for H, X, Y, na in zip(Hs, Xs, Ys, nacts):
        keep = (H.rows < na) & (H.cols < na)
        Hl = oracle.Coo(na, H.rows[keep], H.cols[keep], H.vals[keep])
        np.testing.assert_array_equal(Y.cpu().numpy()[:na], oracle.spmm(Hl, X[:na]))


def test_spmm_batch_rejects_repeated_matrix():
    import paper_1609_01689_gb300 as lob
    rng = np.random.default_rng(3)
    H = random_upper(100, 0.1, rng)
    M = lob.Matrix(100, H.rows, H.cols, H.vals)
    X = rng.standard_normal((100, 4))
    with pytest.raises(lob.LobError):
        lob.spmm_batch([M, M], [X, X], "fp64")


def _problem(n, seed, nu=30):
    L = synth.layout(n, synth.interp_levels(n), nu, seed)
    r, c, v = synth.generate(L)
    return L, oracle.Coo(n, r, c, v)


# (n, seed, k, nb, mode): sizes and block widths of the serving mix, both arithmetics
MIX = [(1536, 1, 5, 8, "mixed"), (2100, 2, 3, 4, "fp64"), (2600, 3, 8, 8, "mixed"), (1800, 4, 1, 1, "mixed"),
       (3000, 5, 2, 2, "fp64"), (2300, 6, 4, 4, "mixed")]


@pytest.fixture(scope="module")
def mix():
    import paper_1609_01689_gb300 as lob
    out = []
    for n, seed, k, nb, mode in MIX:
        L, H = _problem(n, seed)
        lam_ref, _, _, ok = oracle.lanczos(H, k, 1e-13)
        assert ok
        M = lob.Matrix(n, H.rows, H.cols, H.vals, precond_block=32)
        out.append(dict(L=L, H=H, M=M, k=k, nb=nb, mode=mode, lam_ref=lam_ref, n_small=int(synth.level_starts(L)[2])))
    return out


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


@pytest.mark.parametrize("engine", ["lockstep", "shared"])
def test_server_results_match_alone_and_oracle(mix, engine):
    import torch
    import paper_1609_01689_gb300 as lob
    alone = []
    for p in mix:
        lam, X, st, rc = p["M"].solve(p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"])
        assert rc == lob.LOB_OK
        alone.append(lam)
    srv = lob.Server(budget_bytes=8 << 30, max_active=16, engine=engine)
    Xs, ids = [], []
    for p in mix:
        X = torch.empty((p["M"].n, p["nb"]), dtype=torch.float64, device="cuda")
        Xs.append(X)
        ids.append(srv.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"],
                              X_out=X))
    res = {}
    for _ in range(200000):
        srv.progress(wait=True)
        for i in ids:
            if i not in res:
                r = srv.poll(i)
                if r["state"] == lob.REQ_DONE:
                    res[i] = r
        if len(res) == len(ids):
            break
    assert len(res) == len(ids)
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    for p, i, X, lam_alone in zip(mix, ids, Xs, alone):
        r = res[i]
        assert r["rc"] == lob.LOB_OK
        tol_lam = 1e-9 if p["mode"] == "fp64" else 1e-8
        assert _rel(r["lam"], p["lam_ref"][:p["k"]]).max() <= tol_lam
        assert _rel(r["lam"], lam_alone).max() <= 1e-10
        Xh = X.cpu().numpy()[:, :p["k"]]
        nres = oracle.residual_norms(p["H"], Xh, r["lam"])
        assert nres.max() <= 1e-8 * oracle.norm_inf(p["H"])
        assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"]
    # several solves shared SpMM launches
    assert st["finished"] == len(mix)
    assert st["spmm_launches"] < st["spmm_products"]
    assert st["bytes_in_use"] == 0


def test_server_admits_by_memory_while_others_run(mix):
    """A budget that holds two of the solves at a time: the rest wait in the queue, are admitted
    as memory frees up (while other solves are still running), and all finish correctly; a
    request arriving mid-run joins the running ones."""
    import paper_1609_01689_gb300 as lob
    probe = lob.Server(budget_bytes=64 << 30)
    sizes = []
    for p in mix:
        i = probe.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"])
        sizes.append(probe.poll(i)["bytes"])
    probe.close()
    budget = sorted(sizes)[-1] + sorted(sizes)[-2]
    srv = lob.Server(budget_bytes=budget, max_active=8)
    ids = []
    for p in mix[:4]:
        ids.append(srv.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"]))
    res = {}
    late_submitted = False
    for _ in range(400000):
        srv.progress(wait=True)
        st = srv.stats()
        assert st["bytes_in_use"] <= budget
        if not late_submitted and st["admitted"] >= 2:
            for p in mix[4:]:
                ids.append(srv.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True,
                                      n_small=p["n_small"]))
            late_submitted = True
        for i in ids:
            if i not in res:
                r = srv.poll(i)
                if r["state"] == lob.REQ_DONE:
                    res[i] = r
        if late_submitted and len(res) == len(ids):
            break
    st = srv.stats()
    srv.close()
    assert len(res) == len(mix)
    assert st["bytes_peak"] <= budget
    for p, i in zip(mix, ids):
        r = res[i]
        assert r["rc"] == lob.LOB_OK
        tol_lam = 1e-9 if p["mode"] == "fp64" else 1e-8
        assert _rel(r["lam"], p["lam_ref"][:p["k"]]).max() <= tol_lam
    # continuous batching: some solve was admitted while another was still running
    spans = sorted((r["t_admit_ms"], r["t_done_ms"]) for r in res.values())
    assert any(spans[j][0] < spans[j - 1][1] for j in range(1, len(spans)))
    # and some solve waited in the queue for memory
    assert any(r["t_admit_ms"] > r["t_submit_ms"] + 1e-3 for r in res.values())


def test_server_unbatched_mode_same_results(mix):
    import paper_1609_01689_gb300 as lob
    srv = lob.Server(engine="streams")
    ids = [srv.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"])
           for p in mix[:3]]
    res = {}
    for _ in range(200000):
        srv.progress(wait=True)
        for i in ids:
            if i not in res:
                r = srv.poll(i)
                if r["state"] == lob.REQ_DONE:
                    res[i] = r
        if len(res) == len(ids):
            break
    st = srv.stats()
    srv.close()
    assert st["spmm_launches"] == st["spmm_products"]
    for p, i in zip(mix, ids):
        assert res[i]["rc"] == lob.LOB_OK
        assert _rel(res[i]["lam"], p["lam_ref"][:p["k"]]).max() <= (1e-9 if p["mode"] == "fp64" else 1e-8)


@pytest.mark.parametrize("engine", ["lockstep", "shared"])
def test_server_with_the_diagonal_tile_preconditioner(engine):
    """Solves preconditioned on the diagonal 256 x 256 tiles (FOM on the tile store, Section 4.3)
    served together: each result equals the same solve alone (lob_solve, same options) and the
    oracle, at the tolerances of the other serving tests."""
    import paper_1609_01689_gb300 as lob
    probs = []
    for n, seed, k, nb, mode in [(1536, 1, 5, 8, "mixed"), (2600, 3, 4, 8, "fp64"), (2300, 6, 4, 4, "mixed")]:
        L, H = _problem(n, seed)
        lam_ref, _, _, ok = oracle.lanczos(H, k, 1e-13)
        assert ok
        M = lob.Matrix(n, H.rows, H.cols, H.vals, precond_block=256)
        probs.append(dict(H=H, M=M, k=k, nb=nb, mode=mode, lam_ref=lam_ref, n_small=int(synth.level_starts(L)[2])))
    alone = []
    for p in probs:
        lam, _, _, rc = p["M"].solve(p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"])
        assert rc == lob.LOB_OK
        alone.append(lam)
    srv = lob.Server(budget_bytes=8 << 30, max_active=16, engine=engine)
    ids = [srv.submit(p["M"], p["k"], p["nb"], 1e-8, mode=p["mode"], precond=True, n_small=p["n_small"])
           for p in probs]
    res = {}
    for _ in range(200000):
        srv.progress(wait=True)
        for i in ids:
            if i not in res:
                r = srv.poll(i)
                if r["state"] == lob.REQ_DONE:
                    res[i] = r
        if len(res) == len(ids):
            break
    srv.close()
    assert len(res) == len(ids)
    for p, i, lam_alone in zip(probs, ids, alone):
        r = res[i]
        assert r["rc"] == lob.LOB_OK
        assert _rel(r["lam"], p["lam_ref"][:p["k"]]).max() <= (1e-9 if p["mode"] == "fp64" else 1e-8)
        assert _rel(r["lam"], lam_alone).max() <= 1e-10
    # direct solves need factorised blocks: refused for the tile preconditioner
    srv = lob.Server()
    with pytest.raises(lob.LobError):
        srv.submit(probs[0]["M"], 2, 4, 1e-8, precond=True, precond_solve="direct")
    srv.close()


def test_server_rejects_bad_requests(mix):
    import paper_1609_01689_gb300 as lob
    srv = lob.Server(budget_bytes=1 << 20)
    p = mix[0]
    with pytest.raises(lob.LobError):  # cannot ever fit the budget
        srv.submit(p["M"], p["k"], p["nb"], 1e-8)
    srv.close()
    srv = lob.Server()
    with pytest.raises(lob.LobError):  # nb above the server's limit
        srv.submit(p["M"], 4, 32, 1e-8)
    with pytest.raises(lob.LobError):  # k > nb
        srv.submit(p["M"], 5, 4, 1e-8)
    srv.close()
