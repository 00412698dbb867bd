"""lob_rayleigh_ritz_noalloc: the Rayleigh-Ritz step for callers that cannot allocate device
memory (an allocator that owns the device's memory, or a loop where an allocation's device
synchronisation is not acceptable). It must give what the allocating entry point gives, on
consecutive calls that reuse its fixed workspace, allocate nothing, and refuse sizes beyond that
workspace. Collected last so that a run stopping at the first failure has run every other test
first."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def problem(m, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((500, m))
    A = rng.standard_normal((500, 500))
    A = A + A.T
    return Y.T @ A @ Y, Y.T @ Y


# 40: matrices in shared memory; 120: in the fixed workspace; 192: the workspace exactly full
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [40, 120, 192])
def test_noalloc_matches_allocating_entry_point(m, mode):
    import torch
    import paper_1609_01689_gb300 as lob
    theta = torch.empty(m, dtype=torch.float64, device="cuda")
    C = torch.empty((m, m), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call, seed in enumerate((m, m + 1)):  # two calls in a row, different inputs
        G, M = problem(m, seed)
        Gt, Mt = torch.from_numpy(G).cuda(), torch.from_numpy(M).cuda()
        th_ref, C_ref = lob.rayleigh_ritz(Gt, Mt, mode)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        alloc0 = torch.cuda.memory_allocated()
        lob.rayleigh_ritz_noalloc(Gt, Mt, mode, theta=theta, C=C, info=info)
        torch.cuda.synchronize()
        if call > 0:  # the first call may load the kernel's module; later ones must not allocate
            # (free memory may only grow: a stream-ordered pool can trim itself at a synchronisation)
            assert torch.cuda.mem_get_info()[0] >= free0
        assert torch.cuda.memory_allocated() == alloc0
        th, Cn = theta.cpu().numpy(), C.cpu().numpy()
        th_ref, C_ref = th_ref.cpu().numpy(), C_ref.cpu().numpy()
        scale = np.abs(th_ref).max()
        assert np.abs(th - th_ref).max() <= 1e-11 * scale, (call, np.abs(th - th_ref).max())
        assert np.abs(Cn.T @ M @ Cn - np.eye(m)).max() <= 1e-10
        assert np.abs(G @ Cn - M @ Cn * th).max() <= 1e-10 * np.abs(G).max()
        sign = np.sign((Cn * C_ref).sum(axis=0))
        assert np.abs(Cn * sign - C_ref).max() <= 1e-8 * np.abs(C_ref).max()


def test_noalloc_rejects_sizes_beyond_its_workspace():
    import torch
    import paper_1609_01689_gb300 as lob
    G = torch.eye(193, dtype=torch.float64, device="cuda")
    with pytest.raises(lob.LobError) as e:
        lob.rayleigh_ritz_noalloc(G, G)
    assert e.value.code == lob.LOB_ERR_ARG


def test_noalloc_rejects_tensors_it_would_have_to_copy():
    """The binding checks device, dtype, shape and layout instead of copying (which would
    allocate): a wrong tensor is a ValueError before the library is called."""
    import torch
    import paper_1609_01689_gb300 as lob
    G = torch.eye(8, dtype=torch.float64, device="cuda")
    for bad in (G.float(), G.cpu(), G[:, :4], G.t().contiguous()[::2, ::2], torch.eye(8, 9, dtype=torch.float64,
                                                                                        device="cuda")):
        with pytest.raises(ValueError):
            lob.rayleigh_ritz_noalloc(bad, G)
    with pytest.raises(ValueError):
        lob.rayleigh_ritz_noalloc(G, G, theta=torch.empty(7, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        lob.rayleigh_ritz_noalloc(G, G, info=torch.zeros(1, dtype=torch.int64, device="cuda"))
