import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def golden_path(name):
    return os.path.join(GOLDEN, name)


@pytest.fixture(scope="session")
def c1_problem():
    """The n=1536 workload: host COO, its oracle wrapper and ||H||_inf."""
    import oracle
    import synth
    L = synth.config_layout("c1")
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    return dict(L=L, rows=r, cols=c, vals=v, H=H, normH=oracle.norm_inf(H))


@pytest.fixture(scope="session")
def c1_dense_eig(c1_problem):
    """All eigenpairs of the n=1536 workload by the dense oracle (Householder + QL)."""
    import oracle
    w, Z = oracle.syev(oracle.dense(c1_problem["H"]))
    return w, Z
