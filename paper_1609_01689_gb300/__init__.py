"""Python binding of liblob.so, the GB300 block eigensolver (C ABI in include/lob.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. PyTorch provides device memory and the current stream. There is no CPU path:
if the library is missing, importing the binding raises.

Main objects:
  Matrix(n, rows, cols, vals, precond_block=0)  tile store of the upper triangle (lob_create)
  Matrix.spmm(X, mode)                          Y = H X (lob_spmm)
  Matrix.solve(k, nb, tol, ...)                 k smallest eigenpairs by LOBPCG (lob_solve)
  gram, lincomb, rayleigh_ritz, Matrix.precond_apply   the pieces of one iteration
  spmm_batch(mats, Xs, modes)                   products of several matrices in shared launches
  Server(budget_bytes, max_active)              continuous batching of solves (lob_server_*)
  Batch(problems).solve(k, nb, tol, ...)        many small solves in one persistent schedule (lob_batch_*)
  VMatrix(n, rows, cols, vals, groups, beta)    variable-size blocks with 8 + 8-bit offsets (lob_v*)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))

LOB_OK = 0
LOB_ERR_ARG = -1
LOB_ERR_NOMEM = -2
LOB_ERR_CUDA = -3
LOB_ERR_NOCONV = -4
LOB_ERR_BREAKDOWN = -5

VALUES_FP64, VALUES_FP32, VALUES_BOTH = 1, 2, 3
SPMM_FP64, SPMM_MIXED, SPMM_DF64 = 0, 1, 2
MODE_FP64, MODE_MIXED = 0, 1
PSOLVE_FOM, PSOLVE_DIRECT, PSOLVE_MINRES, PSOLVE_ABS = 0, 1, 2, 3
_PSOLVE = {"fom": 0, "direct": 1, "minres": 2, "abs": 3, 0: 0, 1: 1, 2: 2, 3: 3}
_MODES = {"fp64": 0, "mixed": 1, "df64": 2, "tc": 3, 0: 0, 1: 1, 2: 2, 3: 3}
_ARITH = {"fp64": 0, "df": 1, 0: 0, 1: 1}

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


class Coo(ctypes.Structure):
    _fields_ = [("n", _I64), ("nnz", _I64), ("row", _P), ("col", _P), ("val", _P), ("on_device", _I32)]


class CreateOpts(ctypes.Structure):
    _fields_ = [("tile", _I32), ("values", _I32), ("precond_block", _I32), ("wait_log2", _I32), ("stream", _P)]


class MatrixInfo(ctypes.Structure):
    _fields_ = [("n", _I64), ("nnz", _I64), ("ntiles", _I64), ("n_tile_rows", _I64), ("tile", _I32),
                ("values", _I32), ("precond_block", _I32), ("perm_chunk", _I32), ("norm_inf", _D),
                ("store_bytes", _I64), ("precond_bytes", _I64)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", _I32), ("precond", _I32), ("max_iter", _I32), ("refine_iter", _I32), ("norm_H", _D),
                ("n_small", _I64), ("seed", ctypes.c_uint64), ("precond_shift", _I32), ("precond_solve", _I32),
                ("precond_steps", _I32), ("verbose", _I32), ("mixed_tol", _D), ("stream", _P),
                ("n_small_inner", _I64), ("guess_tol", _D), ("rr_arith", _I32), ("refine_arith", _I32),
                ("guess_correct", _I32), ("reserved2", _I32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", _I32), ("refine_iterations", _I32), ("spmm_calls", _I32), ("restarts", _I32),
                ("precond_dropped", _I32), ("reserved", _I32), ("time_ms", _D), ("phase_ms", _D * 8), ("spmm_bytes", _D), ("spmm_calls_mode", _I32 * 4),
                ("spmm_ms_mode", _D * 4), ("spmm_bytes_mode", _D * 4), ("residual", _D * 64),
                ("guess_relres", _D * 2)]

    PHASES = ("spmm", "gram", "rr", "update", "precond", "residual", "orth", "guess")

    def to_dict(self, nb):
        return dict(iterations=self.iterations, refine_iterations=self.refine_iterations,
                    spmm_calls=self.spmm_calls, restarts=self.restarts, precond_dropped=self.precond_dropped,
                    time_ms=self.time_ms,
                    phase_ms={p: self.phase_ms[i] for i, p in enumerate(self.PHASES)},
                    spmm_bytes=self.spmm_bytes,
                    spmm_by_mode={m: dict(calls=self.spmm_calls_mode[i], ms=self.spmm_ms_mode[i],
                                          bytes=self.spmm_bytes_mode[i])
                                  for i, m in enumerate(("fp64", "mixed", "df64"))},
                    residual=[self.residual[j] for j in range(nb)],
                    guess_relres=[self.guess_relres[0], self.guess_relres[1]])


class LanczosStats(ctypes.Structure):
    _fields_ = [("steps", _I32), ("reserved", _I32), ("time_ms", _D), ("spmv_ms", _D), ("device_bytes", _D)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_active", _I32), ("engine", _I32)]


ENGINE_LOCKSTEP, ENGINE_SHARED, ENGINE_STREAMS = 0, 1, 2
_ENGINES = {"lockstep": 0, "shared": 1, "streams": 2, 0: 0, 1: 1, 2: 2}


class Request(ctypes.Structure):
    _fields_ = [("H", _P), ("k", _I32), ("nb", _I32), ("tol", _D), ("X", _P), ("opts", SolveOpts)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE = 1, 2, 3


class Result(ctypes.Structure):
    _fields_ = [("state", _I32), ("rc", _I32), ("lambda_", _D * 16), ("stats", Stats), ("t_submit_ms", _D),
                ("t_admit_ms", _D), ("t_done_ms", _D), ("bytes", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _I64), ("admitted", _I64), ("finished", _I64), ("active", _I64), ("queued", _I64),
                ("bytes_in_use", ctypes.c_uint64), ("bytes_peak", ctypes.c_uint64), ("spmm_launches", _I64),
                ("spmm_products", _I64), ("progress_calls", _I64), ("rounds", _I64), ("host_ms", _D),
                ("wait_ms", _D)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("k", _I32), ("nb", _I32), ("mode", _I32), ("max_iter", _I32), ("tol", _D), ("mixed_tol", _D),
                ("seed", ctypes.c_uint64), ("tile", _I32), ("threads", _I32), ("per_sm", _I32),
                ("tune_iter", _I32), ("stream", _P)]


class BatchStats(ctypes.Structure):
    _fields_ = [("tile", _I32), ("threads", _I32), ("per_sm", _I32), ("candidates", _I32), ("tune_ms", _D),
                ("kernel_ms", _D), ("wall_ms", _D), ("rows", _I64), ("entries", _I64), ("work_bytes", _I64)]


class VMatrixInfo(ctypes.Structure):
    _fields_ = [("n", _I64), ("nnz", _I64), ("nblocks", _I64), ("ntiles", _I64), ("beta_max", _I32),
                ("reserved", _I32), ("store_bytes", _I64), ("kernel_bytes", _I64)]


class LobError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


def _load():
    path = os.path.join(_HERE, "liblob.so")
    if not os.path.exists(path):
        raise ImportError(f"liblob.so is not built ({path}); run paper_1609_01689_gb300._build.build()")
    L = ctypes.CDLL(path)
    L.lob_create.argtypes = [ctypes.POINTER(Coo), ctypes.POINTER(CreateOpts), ctypes.POINTER(_P)]
    L.lob_destroy.argtypes = [_P]
    L.lob_matrix_info_get.argtypes = [_P, ctypes.POINTER(MatrixInfo)]
    L.lob_export_tiles.argtypes = [_P, _P, _P, _P, _P, _P, _P]
    L.lob_export_perm.argtypes = [_P, _P]
    L.lob_spmm.argtypes = [_P, _I32, _P, _P, _I32, _P]
    L.lob_check.argtypes = [_P, _P]
    L.lob_gram.argtypes = [_I64, _I32, _P, _I32, _I32, _P, _I32, _P, _I32, _P]
    L.lob_lincomb.argtypes = [_I64, _I32, _P, _I32, _I32, _P, _P, _I32, _I32, _P]
    L.lob_precond_apply.argtypes = [_P, _P, _P, _P, _I32, _I32, _I32, _P]
    L.lob_rayleigh_ritz.argtypes = [_I32, _P, _P, _P, _P, _P, _I32, _P]
    L.lob_rayleigh_ritz_noalloc.argtypes = [_I32, _P, _P, _P, _P, _P, _I32, _P]
    L.lob_rayleigh_ritz_noalloc.restype = ctypes.c_int
    L.lob_solve.argtypes = [_P, _I32, _I32, _D, _P, ctypes.POINTER(SolveOpts), _P, _P, ctypes.POINTER(Stats)]
    L.lob_spmm_batch.argtypes = [_I32, _P, _P, _P, _P, _P, _P, _P]
    L.lob_lanczos.argtypes = [_P, _I32, _D, _I32, _I32, ctypes.c_uint64, _P, _P, ctypes.POINTER(LanczosStats), _P]
    L.lob_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(_P)]
    L.lob_server_submit.argtypes = [_P, ctypes.POINTER(Request), ctypes.POINTER(_I64)]
    L.lob_server_progress.argtypes = [_P, _I32, ctypes.POINTER(_I32)]
    L.lob_server_poll.argtypes = [_P, _I64, ctypes.POINTER(Result)]
    L.lob_server_stats_get.argtypes = [_P, ctypes.POINTER(ServerStats)]
    L.lob_server_destroy.argtypes = [_P]
    L.lob_batch_create.argtypes = [_I32, _P, _P, ctypes.POINTER(_P)]
    L.lob_batch_destroy.argtypes = [_P]
    L.lob_batch_solve.argtypes = [_P, ctypes.POINTER(BatchOpts), _P, _P, _P, _P, ctypes.POINTER(BatchStats)]
    L.lob_vcreate.argtypes = [ctypes.POINTER(Coo), _P, _I32, _I32, _P, ctypes.POINTER(_P)]
    L.lob_vdestroy.argtypes = [_P]
    L.lob_vinfo.argtypes = [_P, ctypes.POINTER(VMatrixInfo)]
    L.lob_vexport.argtypes = [_P, _P, _P, _P, _P, _P, _P]
    L.lob_vspmm.argtypes = [_P, _P, _P, _I32, _P]
    L.lob_kernel_launches.argtypes = []
    L.lob_kernel_launches.restype = ctypes.c_longlong
    L.lob_strerror.argtypes = [ctypes.c_int]
    L.lob_strerror.restype = ctypes.c_char_p
    for f in ("lob_create", "lob_destroy", "lob_matrix_info_get", "lob_export_tiles", "lob_export_perm", "lob_spmm",
              "lob_check", "lob_gram",
              "lob_lincomb", "lob_precond_apply", "lob_rayleigh_ritz", "lob_solve", "lob_spmm_batch", "lob_lanczos",
              "lob_server_create", "lob_server_submit", "lob_server_progress", "lob_server_poll",
              "lob_server_stats_get", "lob_server_destroy", "lob_batch_create", "lob_batch_destroy",
              "lob_batch_solve", "lob_vcreate", "lob_vdestroy", "lob_vinfo", "lob_vexport", "lob_vspmm"):
        getattr(L, f).restype = ctypes.c_int
    return L


_lib = None


def lib():
    """The loaded liblob.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def build(force=False):
    """Compile liblob.so for sm_103a (nvcc) and load it."""
    global _lib
    _build.build(force=force)
    _lib = None
    return lib()


def kernel_launches():
    """Kernels this library has launched in this process (lob_kernel_launches)."""
    return int(lib().lob_kernel_launches())


def strerror(code):
    return lib().lob_strerror(code).decode()


def _check(rc, what):
    if rc != LOB_OK:
        raise LobError(rc, what)


def _torch():
    import torch
    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dev_f64(x):
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(device="cuda", dtype=torch.float64)
    return x.contiguous()


class Matrix:
    """Device tile store of a symmetric H given by its upper triangle (lob_create)."""

    def __init__(self, n, rows, cols, vals, precond_block=0, values=VALUES_BOTH, wait_log2=0):
        torch = _torch()
        self._keep = []
        if isinstance(rows, np.ndarray):
            r = np.ascontiguousarray(rows, dtype=np.int64)
            c = np.ascontiguousarray(cols, dtype=np.int64)
            v = np.ascontiguousarray(vals, dtype=np.float64)
            coo = Coo(n, len(r), r.ctypes.data, c.ctypes.data, v.ctypes.data, 0)
            self._keep += [r, c, v]
        else:
            r = rows.to(device="cuda", dtype=torch.int64).contiguous()
            c = cols.to(device="cuda", dtype=torch.int64).contiguous()
            v = vals.to(device="cuda", dtype=torch.float64).contiguous()
            coo = Coo(n, r.numel(), r.data_ptr(), c.data_ptr(), v.data_ptr(), 1)
            self._keep += [r, c, v]
        opts = CreateOpts(0, values, precond_block, wait_log2, _stream())
        h = _P()
        _check(lib().lob_create(ctypes.byref(coo), ctypes.byref(opts), ctypes.byref(h)), "lob_create")
        self._h = h
        self._keep = []
        self.n = int(n)

    def close(self):
        if getattr(self, "_h", None):
            lib().lob_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = MatrixInfo()
        _check(lib().lob_matrix_info_get(self._h, ctypes.byref(inf)), "lob_matrix_info_get")
        return {f: getattr(inf, f) for f, _ in MatrixInfo._fields_}

    def export_tiles(self):
        inf = self.info()
        nt, ntl, nnz = inf["n_tile_rows"], inf["ntiles"], inf["nnz"]
        rp = np.empty(nt + 1, np.int64)
        tc = np.empty(ntl, np.int32)
        tp = np.empty(ntl + 1, np.int64)
        rc = np.empty(nnz, np.uint32)
        v64 = np.empty(nnz, np.float64) if inf["values"] & VALUES_FP64 else None
        v32 = np.empty(nnz, np.float32) if inf["values"] & VALUES_FP32 else None
        _check(lib().lob_export_tiles(self._h, rp.ctypes.data, tc.ctypes.data, tp.ctypes.data, rc.ctypes.data,
                                      v64.ctypes.data if v64 is not None else None,
                                      v32.ctypes.data if v32 is not None else None), "lob_export_tiles")
        return dict(tile_rowptr=rp, tile_col=tc, tile_ptr=tp, rc=rc, v64=v64, v32=v32, ntiles=ntl)

    def export_perm(self):
        """The kernel-private column-order permutation (lob_export_perm)."""
        perm = np.empty(self.info()["nnz"], np.uint16)
        _check(lib().lob_export_perm(self._h, perm.ctypes.data), "lob_export_perm")
        return perm

    def spmm(self, X, mode="fp64", out=None):
        X = _dev_f64(X)
        nb = 1 if X.dim() == 1 else X.shape[1]
        Y = out if out is not None else _torch().empty_like(X)
        _check(lib().lob_spmm(self._h, _MODES[mode], X.data_ptr(), Y.data_ptr(), nb, _stream()), "lob_spmm")
        return Y

    def check(self):
        """Raise LobError if an SpMM kernel on this matrix gave up on a bounded wait (lob_check)."""
        _check(lib().lob_check(self._h, _stream()), "lob_check")

    def precond_apply(self, mu, R, solve="direct", steps=3):
        """Approximate solves of eq. 11 per block and column (lob_precond_apply)."""
        R = _dev_f64(R)
        mu = _dev_f64(mu)
        W = _torch().empty_like(R)
        _check(lib().lob_precond_apply(self._h, mu.data_ptr(), R.data_ptr(), W.data_ptr(), R.shape[1],
                                       _PSOLVE[solve], steps, _stream()), "lob_precond_apply")
        return W

    def solve(self, k, nb, tol, X0=None, mode="fp64", precond=False, n_small=0, max_iter=0, refine_iter=0,
              seed=1, precond_shift=0, mixed_tol=0.0, norm_H=0.0, X_out=None, precond_solve="fom", precond_steps=3,
              stats=True, n_small_inner=0, guess_tol=0.0, rr_arith="fp64", refine_arith="fp64",
              guess_correct=False):
        """k smallest eigenpairs (lob_solve). Returns (lam, X, stats, status). stats=False passes no
        stats struct: the solver then keeps no phase timers and replays its stages as CUDA graphs."""
        torch = _torch()
        X = X_out if X_out is not None else torch.empty((self.n, nb), dtype=torch.float64, device="cuda")
        x0 = _dev_f64(X0) if X0 is not None else None
        lam = np.zeros(k, np.float64)
        st = Stats()
        o = SolveOpts(_MODES[mode], int(bool(precond)), max_iter, refine_iter, norm_H, n_small, seed, precond_shift,
                      _PSOLVE[precond_solve], precond_steps, 0, mixed_tol, _stream(), n_small_inner, guess_tol,
                      _ARITH[rr_arith], _ARITH[refine_arith], int(bool(guess_correct)), 0)
        rc = lib().lob_solve(self._h, k, nb, tol, x0.data_ptr() if x0 is not None else None, ctypes.byref(o),
                             lam.ctypes.data, X.data_ptr(), ctypes.byref(st) if stats else None)
        if rc not in (LOB_OK, LOB_ERR_NOCONV):
            raise LobError(rc, "lob_solve")
        return lam, X, st.to_dict(nb), rc


def lanczos(matrix, k, tol, max_steps=1000, check=10, seed=7, vectors=True):
    """k smallest eigenpairs by the GPU Lanczos baseline (lob_lanczos). Returns (lam, X, stats, rc)."""
    torch = _torch()
    lam = np.zeros(k, np.float64)
    X = torch.empty((matrix.n, k), dtype=torch.float64, device="cuda") if vectors else None
    st = LanczosStats()
    rc = lib().lob_lanczos(matrix.handle, k, tol, max_steps, check, seed, lam.ctypes.data,
                           X.data_ptr() if X is not None else None, ctypes.byref(st), _stream())
    if rc not in (LOB_OK, LOB_ERR_NOCONV):
        raise LobError(rc, "lob_lanczos")
    return lam, X, dict(steps=st.steps, time_ms=st.time_ms, spmv_ms=st.spmv_ms, device_bytes=st.device_bytes), rc


def gram(A, B, mode="fp64"):
    """A^T B for tall-skinny device blocks (lob_gram)."""
    A = _dev_f64(A); B = _dev_f64(B)
    G = _torch().empty((A.shape[1], B.shape[1]), dtype=_torch().float64, device="cuda")
    _check(lib().lob_gram(A.shape[0], A.shape[1], A.data_ptr(), A.shape[1], B.shape[1], B.data_ptr(), B.shape[1],
                          G.data_ptr(), _MODES[mode], _stream()), "lob_gram")
    return G


def lincomb(A, C, mode="fp64"):
    """A C for a tall-skinny device block (lob_lincomb)."""
    A = _dev_f64(A); C = _dev_f64(C)
    Y = _torch().empty((A.shape[0], C.shape[1]), dtype=_torch().float64, device="cuda")
    _check(lib().lob_lincomb(A.shape[0], A.shape[1], A.data_ptr(), A.shape[1], C.shape[1], C.data_ptr(), Y.data_ptr(),
                             C.shape[1], _MODES[mode], _stream()), "lob_lincomb")
    return Y


def rayleigh_ritz(G, M, mode="fp64"):
    """theta, C with G C = M C diag(theta) (lob_rayleigh_ritz); raises on an indefinite M."""
    torch = _torch()
    G = _dev_f64(G); M = _dev_f64(M)
    m = G.shape[0]
    theta = torch.empty(m, dtype=torch.float64, device="cuda")
    C = torch.empty((m, m), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib().lob_rayleigh_ritz(m, G.data_ptr(), M.data_ptr(), theta.data_ptr(), C.data_ptr(), info.data_ptr(),
                                   _MODES[mode], _stream()), "lob_rayleigh_ritz")
    if int(info.item()) != 0:
        raise np.linalg.LinAlgError(f"Gram matrix not positive definite (pivot {int(info.item())})")
    return theta, C


def _need(x, name, shape, dtype):
    """Reject (never copy) a tensor the no-allocation entry point cannot take as it is."""
    if not (hasattr(x, "is_cuda") and x.is_cuda and x.dtype == dtype and tuple(x.shape) == shape
            and x.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous {dtype} CUDA tensor of shape {shape}")


def rayleigh_ritz_noalloc(G, M, mode="fp64", theta=None, C=None, info=None):
    """rayleigh_ritz through lob_rayleigh_ritz_noalloc: the library allocates no device memory
    (its workspace is a fixed array for m <= 192). The caller may pass preallocated output
    tensors; G and M must already be square, contiguous FP64 device tensors. Inputs that do not
    fit are rejected with ValueError rather than copied, so the call itself allocates nothing."""
    torch = _torch()
    m = G.shape[0]
    _need(G, "G", (m, m), torch.float64)
    _need(M, "M", (m, m), torch.float64)
    theta = theta if theta is not None else torch.empty(m, dtype=torch.float64, device="cuda")
    C = C if C is not None else torch.empty((m, m), dtype=torch.float64, device="cuda")
    info = info if info is not None else torch.zeros(1, dtype=torch.int32, device="cuda")
    _need(theta, "theta", (m,), torch.float64)
    _need(C, "C", (m, m), torch.float64)
    _need(info, "info", (1,), torch.int32)
    _check(lib().lob_rayleigh_ritz_noalloc(m, G.data_ptr(), M.data_ptr(), theta.data_ptr(), C.data_ptr(),
                                           info.data_ptr(), _MODES[mode], _stream()), "lob_rayleigh_ritz_noalloc")
    if int(info.item()) != 0:
        raise np.linalg.LinAlgError(f"Gram matrix not positive definite (pivot {int(info.item())})")
    return theta, C


def spmm_batch(mats, Xs, modes="fp64", n_act=None):
    """[H_j X_j] for distinct matrices in shared launches (lob_spmm_batch); n_act restricts each
    product to the leading n_act[j] block."""
    torch = _torch()
    nj = len(mats)
    if isinstance(modes, (str, int)):
        modes = [modes] * nj
    Xs = [_dev_f64(x) for x in Xs]
    Ys = [torch.empty_like(x) for x in Xs]
    H = (_P * nj)(*[m.handle.value for m in mats])
    Xp = (_P * nj)(*[x.data_ptr() for x in Xs])
    Yp = (_P * nj)(*[y.data_ptr() for y in Ys])
    nb = (_I32 * nj)(*[1 if x.dim() == 1 else x.shape[1] for x in Xs])
    md = (_I32 * nj)(*[_MODES[m] for m in modes])
    na = (_I64 * nj)(*n_act) if n_act is not None else None
    _check(lib().lob_spmm_batch(nj, H, Xp, Yp, nb, md, na, _stream()), "lob_spmm_batch")
    return Ys


class Server:
    """Continuous batching of eigen-solves (lob_server_*): submit() queues a solve, progress()
    admits what fits the device-memory budget and advances every admitted solve, sharing the
    SpMM launches; poll() returns a finished solve's eigenvalues, stats and timestamps."""

    def __init__(self, budget_bytes=0, max_active=0, engine="lockstep"):
        o = ServerOpts(budget_bytes, max_active, _ENGINES[engine])
        h = _P()
        _check(lib().lob_server_create(ctypes.byref(o), ctypes.byref(h)), "lob_server_create")
        self._h = h
        self._keep = {}

    def submit(self, matrix, k, nb, tol, mode="mixed", precond=False, n_small=0, max_iter=0, refine_iter=0, seed=1,
               precond_shift=0, mixed_tol=0.0, X_out=None, precond_solve="fom", precond_steps=3, rr_arith="fp64",
               refine_arith="fp64"):
        o = SolveOpts(_MODES[mode], int(bool(precond)), max_iter, refine_iter, 0.0, n_small, seed, precond_shift,
                      _PSOLVE[precond_solve], precond_steps, 0, mixed_tol, None, 0, 0.0, _ARITH[rr_arith],
                      _ARITH[refine_arith])
        r = Request(matrix.handle, k, nb, tol, X_out.data_ptr() if X_out is not None else None, o)
        rid = _I64()
        _check(lib().lob_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), "lob_server_submit")
        self._keep[rid.value] = (matrix, k)
        return rid.value

    def progress(self, wait=True):
        nd = _I32()
        _check(lib().lob_server_progress(self._h, int(bool(wait)), ctypes.byref(nd)), "lob_server_progress")
        return nd.value

    def poll(self, rid):
        """dict(state, bytes, t_submit_ms, ...); once state == REQ_DONE also rc, lam (k values),
        stats, t_admit_ms, t_done_ms, and the record is released."""
        res = Result()
        _check(lib().lob_server_poll(self._h, rid, ctypes.byref(res)), "lob_server_poll")
        out = dict(state=res.state, bytes=int(res.bytes), t_submit_ms=res.t_submit_ms, t_admit_ms=res.t_admit_ms)
        if res.state == REQ_DONE:
            _, k = self._keep.pop(rid, (None, 16))
            out.update(rc=res.rc, lam=np.array(res.lambda_[:k]), stats=res.stats.to_dict(16),
                       t_done_ms=res.t_done_ms)
        return out

    def stats(self):
        st = ServerStats()
        _check(lib().lob_server_stats_get(self._h, ctypes.byref(st)), "lob_server_stats_get")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().lob_server_destroy(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent small matrices (n <= 65,535 each) solved together by one persistent
    kernel schedule replayed from a CUDA graph (lob_batch_*). problems: a list of (n, rows,
    cols, vals) upper triangles, numpy (host) or torch CUDA tensors (device)."""

    def __init__(self, problems):
        torch = _torch()
        keep = []
        coos = (Coo * len(problems))()
        for i, (n, rows, cols, vals) in enumerate(problems):
            if isinstance(rows, np.ndarray):
                r = np.ascontiguousarray(rows, dtype=np.int64)
                c = np.ascontiguousarray(cols, dtype=np.int64)
                v = np.ascontiguousarray(vals, dtype=np.float64)
                coos[i] = Coo(int(n), len(r), r.ctypes.data, c.ctypes.data, v.ctypes.data, 0)
            else:
                r = rows.to(device="cuda", dtype=torch.int64).contiguous()
                c = cols.to(device="cuda", dtype=torch.int64).contiguous()
                v = vals.to(device="cuda", dtype=torch.float64).contiguous()
                coos[i] = Coo(int(n), r.numel(), r.data_ptr(), c.data_ptr(), v.data_ptr(), 1)
            keep += [r, c, v]
        h = _P()
        _check(lib().lob_batch_create(len(problems), coos, _stream(), ctypes.byref(h)), "lob_batch_create")
        self._h = h
        self.sizes = [int(p[0]) for p in problems]
        self.count = len(problems)
        self.rows = int(sum(self.sizes))
        self.row0 = np.concatenate([[0], np.cumsum(self.sizes)[:-1]]).astype(np.int64)

    def close(self):
        if getattr(self, "_h", None):
            lib().lob_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, k, nb, tol, mode="mixed", max_iter=0, mixed_tol=0.0, seed=1, tile=0, threads=0, per_sm=0,
              tune_iter=0, vectors=False):
        """Solve every instance (lob_batch_solve). Returns (lam [count, k], status [count],
        iters [count, 2], X [rows, nb] or None, stats dict), all numpy except X (torch, device)."""
        torch = _torch()
        lam = torch.empty((self.count, k), dtype=torch.float64, device="cuda")
        status = torch.empty(self.count, dtype=torch.int32, device="cuda")
        iters = torch.empty((self.count, 2), dtype=torch.int32, device="cuda")
        X = torch.empty((self.rows, nb), dtype=torch.float64, device="cuda") if vectors else None
        o = BatchOpts(k, nb, _MODES[mode], max_iter, tol, mixed_tol, seed, tile, threads, per_sm, tune_iter,
                      _stream())
        st = BatchStats()
        _check(lib().lob_batch_solve(self._h, ctypes.byref(o), lam.data_ptr(), status.data_ptr(), iters.data_ptr(),
                                     X.data_ptr() if X is not None else None, ctypes.byref(st)), "lob_batch_solve")
        return (lam.cpu().numpy(), status.cpu().numpy(), iters.cpu().numpy(), X,
                {f: getattr(st, f) for f, _ in BatchStats._fields_})


class VMatrix:
    """Compact block store of the upper triangle: each group [g_i, g_i+1) cut into blocks of at
    most beta_max rows, entries as (r << 8) | c and an FP32 value (lob_vcreate)."""

    def __init__(self, n, rows, cols, vals, group_starts, beta_max=256):
        torch = _torch()
        if isinstance(rows, np.ndarray):
            r = np.ascontiguousarray(rows, dtype=np.int64)
            c = np.ascontiguousarray(cols, dtype=np.int64)
            v = np.ascontiguousarray(vals, dtype=np.float64)
            coo = Coo(n, len(r), r.ctypes.data, c.ctypes.data, v.ctypes.data, 0)
        else:
            r = rows.to(device="cuda", dtype=torch.int64).contiguous()
            c = cols.to(device="cuda", dtype=torch.int64).contiguous()
            v = vals.to(device="cuda", dtype=torch.float64).contiguous()
            coo = Coo(n, r.numel(), r.data_ptr(), c.data_ptr(), v.data_ptr(), 1)
        g = np.ascontiguousarray(group_starts, dtype=np.int64)
        h = _P()
        _check(lib().lob_vcreate(ctypes.byref(coo), g.ctypes.data, len(g), beta_max, _stream(), ctypes.byref(h)),
               "lob_vcreate")
        self._h = h
        self.n = int(n)

    def close(self):
        if getattr(self, "_h", None):
            lib().lob_vdestroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = VMatrixInfo()
        _check(lib().lob_vinfo(self._h, ctypes.byref(inf)), "lob_vinfo")
        return {f: getattr(inf, f) for f, _ in VMatrixInfo._fields_}

    def export(self):
        inf = self.info()
        nblk, ntl, nnz = inf["nblocks"], inf["ntiles"], inf["nnz"]
        bnd = np.empty(nblk + 1, np.int64)
        rp = np.empty(nblk + 1, np.int64)
        tc = np.empty(ntl, np.int32)
        tp = np.empty(ntl + 1, np.int64)
        rc = np.empty(nnz, np.uint16)
        v32 = np.empty(nnz, np.float32)
        _check(lib().lob_vexport(self._h, bnd.ctypes.data, rp.ctypes.data, tc.ctypes.data, tp.ctypes.data,
                                 rc.ctypes.data, v32.ctypes.data), "lob_vexport")
        return dict(bounds=bnd, tile_rowptr=rp, tile_col=tc, tile_ptr=tp, rc16=rc, v32=v32)

    def spmm(self, X, out=None):
        X = _dev_f64(X)
        nb = 1 if X.dim() == 1 else X.shape[1]
        Y = out if out is not None else _torch().empty_like(X)
        _check(lib().lob_vspmm(self._h, X.data_ptr(), Y.data_ptr(), nb, _stream()), "lob_vspmm")
        return Y
