"""Write stored expected values for the large workloads. Calls only oracle/ and synth/.

  c2_eigs.txt: the 10 smallest eigenvalues of the n = 500,000 workload (levels 0..10,
  ~200 nonzeros per row, seed 1) by the oracle's FP64 Lanczos with full reorthogonalisation,
  Ritz residual estimates <= 1e-12 ||H||_inf.
  c3_eigs.txt: the same for the n = 8,000,000 workload (levels 0..14, ~300 nonzeros per row,
  seed 1, 1.2e9 stored entries), through the oracle's CSR form so that the matrix (14 GB) and
  the Lanczos basis fit in host memory together. About an hour on one core.

Usage: python tests/golden/make_golden.py [c2] [c3]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def c2():
    L = synth.config_layout("c2")
    r, c, v = synth.generate(L)
    H = oracle.Coo(L.n, r, c, v)
    nH = oracle.norm_inf(H)
    t0 = time.time()
    lam, X, steps, ok = oracle.lanczos(H, 10, 1e-12, nH, max_steps=3000)
    dt = time.time() - t0
    res = oracle.residual_norms(H, X, lam) / nH
    assert ok
    with open(os.path.join(HERE, "c2_eigs.txt"), "w") as f:
        f.write("# 10 smallest eigenvalues of the n=500000 workload (synth c2, seed 1): oracle FP64 Lanczos,\n")
        f.write(f"# full reorthogonalisation, {steps} steps, {dt:.1f} s single-threaded, ||H||_inf = {nH!r},\n")
        f.write(f"# max explicit relative residual {res.max():.3e}. Written by tests/golden/make_golden.py.\n")
        for x in lam:
            f.write(f"{float(x)!r}\n")
    print(steps, dt, lam, res.max())


def c3():
    L = synth.config_layout("c3")
    t0 = time.time()
    r, c, v = synth.generate(L, copy=False)  # views into the generator's buffers: no second copy
    nH = oracle.norm_inf(oracle.Coo(L.n, r, c, v))
    H = oracle.Csr.from_sorted_coo(L.n, r, c, v)
    nnz = len(v)
    del r, c
    t_gen = time.time() - t0
    t0 = time.time()
    lam, X, steps, ok = oracle.lanczos_csr(H, 10, 1e-12, nH, max_steps=700)
    dt = time.time() - t0
    R = oracle.spmm_csr(H, X) - X * lam[None, :]
    res = np.sqrt((R * R).sum(axis=0)) / nH
    assert ok
    with open(os.path.join(HERE, "c3_eigs.txt"), "w") as f:
        f.write(f"# 10 smallest eigenvalues of the n=8000000 workload (synth c3, seed 1, {nnz} stored entries): oracle\n")
        f.write(f"# FP64 Lanczos, full reorthogonalisation, {steps} steps, {dt:.1f} s single-threaded, ||H||_inf = {nH!r},\n")
        f.write(f"# max explicit relative residual {res.max():.3e}. Written by tests/golden/make_golden.py.\n")
        for x in lam:
            f.write(f"{float(x)!r}\n")
    print(steps, dt, t_gen, lam, res.max())


if __name__ == "__main__":
    which = sys.argv[1:] or ["c2"]
    if "c2" in which:
        c2()
    if "c3" in which:
        c3()
