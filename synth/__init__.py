"""Seeded synthetic Hamiltonians shaped like the paper's nuclear CI matrices.

Input generation only: this module holds none of the eigensolver's arithmetic. The CPU
oracle (``oracle/``) and the CUDA path (``paper_1609_01689_gb300``) both consume it and
share nothing else.

The structure follows Sections 2.1-2.2 of the paper: basis states ordered by truncation
level (graded diagonal, eq. 3), with coupling only between nearby levels, giving a block
banded pattern. The per-entry definition is in ``synth_core.h``; host and device
generators produce the same COO bit for bit.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libsynth_host.so")
_DEV_SO = os.path.join(_HERE, "libsynth_dev.so")
MAX_LEVELS = 32


class Layout(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("Q", ctypes.c_int32),
        ("nu", ctypes.c_int32),
        ("w_min", ctypes.c_int32),
        ("w_div", ctypes.c_int32),
        ("draw_pct", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("start", ctypes.c_int64 * (MAX_LEVELS + 1)),
    ]


def _stale(out: str, srcs: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_host() -> str:
    srcs = [os.path.join(_HERE, f) for f in ("synth_host.c", "synth_core.h", "synth.h")]
    if _stale(_HOST_SO, srcs):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", _HOST_SO, srcs[0]])
    return _HOST_SO


def build_device() -> str:
    srcs = [os.path.join(_HERE, f) for f in ("synth_dev.cu", "synth_core.h", "synth.h")]
    if _stale(_DEV_SO, srcs):
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-shared", "-Xcompiler", "-fPIC", "-o", _DEV_SO, srcs[0]])
    return _DEV_SO


_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        lib = ctypes.CDLL(build_host())
        lib.syn_layout_init.argtypes = [ctypes.POINTER(Layout), ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]
        lib.syn_layout_init.restype = ctypes.c_int
        lib.syn_candidate_cap.argtypes = [ctypes.POINTER(Layout)]
        lib.syn_candidate_cap.restype = ctypes.c_int64
        lib.syn_draws_per_row.argtypes = [ctypes.POINTER(Layout)]
        lib.syn_draws_per_row.restype = ctypes.c_int64
        lib.syn_generate_host.argtypes = [ctypes.POINTER(Layout), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64]
        lib.syn_generate_host.restype = ctypes.c_int64
        _host = lib
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        lib = ctypes.CDLL(build_device())
        lib.syn_generate_device.argtypes = [ctypes.POINTER(Layout), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.syn_generate_device.restype = ctypes.c_int64
        _dev = lib
    return _dev


def interp_levels(n: int) -> int:
    """Number of the top level Q for sizes between the named workloads: linear in log n
    through (1536, 6), (5e5, 10), (8e6, 14), clamped to [6, 14]."""
    pts = [(math.log(1536), 6.0), (math.log(5e5), 10.0), (math.log(8e6), 14.0)]
    x = math.log(max(n, 2))
    if x <= pts[0][0]:
        q = pts[0][1] + (x - pts[0][0]) * (pts[1][1] - pts[0][1]) / (pts[1][0] - pts[0][0])
    elif x <= pts[1][0]:
        q = pts[0][1] + (x - pts[0][0]) * (pts[1][1] - pts[0][1]) / (pts[1][0] - pts[0][0])
    else:
        q = pts[1][1] + (x - pts[1][0]) * (pts[2][1] - pts[1][1]) / (pts[2][0] - pts[1][0])
    return int(min(14, max(6, round(q))))


def layout(n: int, Q: int, nu: int, seed: int, w_min: int = 64, w_div: int = 0, draw_pct: int = 0) -> Layout:
    """draw_pct: draws per row in percent of nu (0 = 60)."""
    L = Layout()
    rc = _host_lib().syn_layout_init(ctypes.byref(L), n, Q, nu, w_min, w_div, seed)
    if rc != 0 or draw_pct < 0:
        raise ValueError(f"bad generator parameters n={n} Q={Q} nu={nu} w_min={w_min} w_div={w_div}")
    L.draw_pct = draw_pct
    return L


def level_starts(L: Layout) -> np.ndarray:
    return np.array([L.start[q] for q in range(L.Q + 2)], dtype=np.int64)


def candidate_cap(L: Layout) -> int:
    return int(_host_lib().syn_candidate_cap(ctypes.byref(L)))


def generate(L: Layout, copy: bool = True):
    """Host COO (rows, cols, vals) of the upper triangle incl. diagonal, sorted by (row, col).
    copy=False returns views into the generator's candidate-sized buffers (no second copy of a
    large matrix; the buffers' unused tails stay allocated)."""
    cap = candidate_cap(L)
    rows = np.empty(cap, dtype=np.int64)
    cols = np.empty(cap, dtype=np.int64)
    vals = np.empty(cap, dtype=np.float64)
    nnz = _host_lib().syn_generate_host(ctypes.byref(L), rows.ctypes.data, cols.ctypes.data, vals.ctypes.data, cap)
    if nnz < 0:
        raise MemoryError(f"host generator failed ({nnz})")
    if not copy:
        return rows[:nnz], cols[:nnz], vals[:nnz]
    return rows[:nnz].copy(), cols[:nnz].copy(), vals[:nnz].copy()


def generate_device(L: Layout, device: str = "cuda", stream: int = 0):
    """Device COO as torch tensors (rows, cols, vals); identical to :func:`generate`."""
    import torch

    cap = candidate_cap(L)
    rows = torch.empty(cap, dtype=torch.int64, device=device)
    cols = torch.empty(cap, dtype=torch.int64, device=device)
    vals = torch.empty(cap, dtype=torch.float64, device=device)
    nnz = _dev_lib().syn_generate_device(ctypes.byref(L), rows.data_ptr(), cols.data_ptr(), vals.data_ptr(), cap,
                                         ctypes.c_void_p(stream))
    if nnz < 0:
        raise RuntimeError(f"device generator failed ({nnz})")
    return rows[:nnz], cols[:nnz], vals[:nnz]


# Workload shapes. Sizes, level counts, nonzeros per row, block sizes and seeds of the
# five workloads: a plain FP64 solve (C1), the precision study (C2), the large single
# solve (C3), serving (C4) and batched small instances (C5).
CONFIGS = {
    "c1": dict(n=1536, Q=6, nu=30, k=5, nb=8, bp=32, seed=1),
    "c2": dict(n=500_000, Q=10, nu=200, k=8, nb=16, bp=32, seed=1),
    # 0.7 nu draws per row: at nu = 300 more draws coincide inside the +-64 bands, and 0.6 nu would
    # leave 269 entries per full row (1.08e9 stored) instead of ~300 (1.20e9)
    "c3": dict(n=8_000_000, Q=14, nu=300, k=10, nb=16, bp=64, seed=1, draw_pct=70),
}


def config_layout(name: str, seed: int | None = None, **over) -> Layout:
    c = dict(CONFIGS[name])
    c.update(over)
    return layout(c["n"], c["Q"], c["nu"], c["seed"] if seed is None else seed, draw_pct=c.get("draw_pct", 0))
