"""lob_rayleigh_ritz_noalloc: the Rayleigh-Ritz step for callers that cannot allocate device
memory (an allocator that owns the device's memory, or a loop where an allocation's device
synchronisation is not acceptable). It must give what the allocating entry point gives, on
consecutive calls that reuse its fixed workspace, and refuse sizes beyond that workspace.
Collected last so that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def problem(m, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((500, m))
    A = rng.standard_normal((500, 500))
    A = A + A.T
    return Y.T @ A @ Y, Y.T @ Y


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [40, 120])  # 40: matrices in shared memory; 120: in the fixed workspace
def test_noalloc_matches_allocating_entry_point(m, mode):
    import torch
    import paper_1609_01689_gb300 as lob
    for call, seed in enumerate((m, m + 1)):  # two calls in a row, different inputs
        G, M = problem(m, seed)
        Gt, Mt = torch.from_numpy(G).cuda(), torch.from_numpy(M).cuda()
        th_ref, C_ref = lob.rayleigh_ritz(Gt, Mt, mode)
        th, C = lob.rayleigh_ritz_noalloc(Gt, Mt, mode)
        th, C, th_ref, C_ref = th.cpu().numpy(), C.cpu().numpy(), th_ref.cpu().numpy(), C_ref.cpu().numpy()
        scale = np.abs(th_ref).max()
        assert np.abs(th - th_ref).max() <= 1e-11 * scale, (call, np.abs(th - th_ref).max())
        assert np.abs(C.T @ M @ C - np.eye(m)).max() <= 1e-10
        assert np.abs(G @ C - M @ C * th).max() <= 1e-10 * np.abs(G).max()
        sign = np.sign((C * C_ref).sum(axis=0))
        assert np.abs(C * sign - C_ref).max() <= 1e-8 * np.abs(C_ref).max()


def test_noalloc_rejects_sizes_beyond_its_workspace():
    import torch
    import paper_1609_01689_gb300 as lob
    G = torch.eye(193, dtype=torch.float64, device="cuda")
    with pytest.raises(lob.LobError) as e:
        lob.rayleigh_ritz_noalloc(G, G)
    assert e.value.code == lob.LOB_ERR_ARG
