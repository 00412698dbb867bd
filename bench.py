#!/usr/bin/env python
"""Benchmark: time to the k smallest eigenpairs with the preconditioned block LOBPCG.

Workload (default): the large single solve -- n = 8,000,000, levels 0..14 with sizes ~2.2^q,
graded diagonal 10 q + U(-1,1), ~300 nonzeros per row coupling levels |dq| <= 2 (1.2e9 stored
upper-triangle entries), seed 1 -- k = 10, nb = 16, block-diagonal preconditioner with 64 x 64
blocks, initial guess from the leading levels {0, 1} (eq. 12), residual tolerance 1e-8 ||H||.
One step = one complete mixed-precision solve (every row of the hot path: SpMM, Gram,
Rayleigh-Ritz, update, residual, preconditioner, initial guess, FP64 refinement) with the matrix
already resident in HBM. --workload c2 runs the n = 500,000 precision study instead.

Prints one JSON line. Also reported: SpMM effective HBM bandwidth against the measured peak
(roofline), the plain FP64 solver's time on the same workload, eigenvalue error against the
FP64 oracle, an end-to-end time from host buffers, and the oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): independent replicas, one seeded instance per rank ("replicas only").
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "c2": dict(name="n=500000 levels 0..10, ~200 nnz/row, k=8, nb=16, preconditioner on the diagonal 256x256 "
                    "tiles (FOM 3), tol 1e-8", cfg="c2", k=8, nb=16, bp=256, tol=1e-8),
    "c1": dict(name="n=1536 levels 0..6, ~30 nnz/row, k=5, nb=8, b_p=32, tol 1e-8", cfg="c1", k=5, nb=8, bp=32,
               tol=1e-8),
    "c3": dict(name="n=8000000 levels 0..14, ~300 nnz/row (1.2e9 stored), k=10, nb=16, b_p=64, tol 1e-8", cfg="c3",
               k=10, nb=16, bp=64, tol=1e-8),
}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) of one FP32-value SpMM launch (k_spmm_ring<16>, parity-ordered
# segments), from one-pass ncu captures of this bench's own runs: n = 500,000 from the kernel mode
# (one launch: 761.0 MB read + 146.2 MB written); n = 8,000,000 from the solve (median over the 29
# full-grid launches among the first 45 of the kernel, 20.49 GB). Valid for the kernel as captured;
# reset to None when the kernel changes.
SPMM_TRAFFIC = {"c2": 907_210_000, "c3": 20_485_000_000}
# Nominal FP64 rate of one GB300 (FLOP/s): the bound of the FP64-value SpMM, which the FP64 pipe
# limits (64 FP64 flops per stored entry at nb = 16).
FP64_NOMINAL_FLOPS = 1.25e12


def golden_eigs(cfg):
    """Stored oracle eigenvalues of a workload and the header facts of their run: (values, steps,
    seconds), or (None, None, None)."""
    path = os.path.join(ROOT, "tests", "golden", f"{cfg}_eigs.txt")
    if not os.path.exists(path):
        return None, None, None
    vals, steps, secs = [], None, None
    for line in open(path):
        if line.startswith("#"):
            if " steps" in line:
                try:
                    steps = int(line.split(" steps")[0].split(",")[-1].strip())
                    secs = float(line.split(" steps,")[1].split(" s ")[0].strip())
                except (ValueError, IndexError):
                    pass
            continue
        if line.strip():
            vals.append(float(line))
    return np.array(vals), steps, secs


_ORACLE_H = {}
_HOST_COO = {}


def host_coo(cfg, layout, dev=None):
    """The workload's upper-triangle COO on the host (once per configuration and seed): copied from
    the device generator's output when given (pinned host memory), else the host generator."""
    import synth

    key = (cfg, int(layout.seed))
    if key not in _HOST_COO:
        if dev is not None:
            import torch
            out = []
            for t in dev:
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t)
                out.append(h)
            _HOST_COO[key] = tuple(out)
        else:
            _HOST_COO[key] = tuple(synth.generate(layout, copy=False))
    return _HOST_COO[key]


def _np(a):
    return a.numpy() if hasattr(a, "numpy") else a


# Oracle Lanczos steps of the two timed sample runs per workload (each run is a complete oracle
# Lanczos call of that many steps; about 10-30 s of CPU work together on one core).
ORACLE_SAMPLE_STEPS = {"c1": (10, 30), "c2": (10, 30), "c3": (2, 5)}


def oracle_matrix(cfg, layout, dev=None):
    """The workload in the oracle's CSR form (the COO form's arithmetic; fits beside the Lanczos
    basis at 1.2e9 entries) and its ||H||_inf, built once per configuration and seed."""
    import oracle

    key = (cfg, int(layout.seed))
    if key not in _ORACLE_H:
        r, c, v = (_np(a) for a in host_coo(cfg, layout, dev))
        nH = oracle.norm_inf(oracle.Coo(layout.n, r, c, v))
        _ORACLE_H[key] = (oracle.Csr.from_sorted_coo(layout.n, r, c, v), nH)
    return _ORACLE_H[key]


def oracle_run_s(H, nH, steps):
    """Seconds of one oracle Lanczos call of the given number of steps."""
    import oracle

    t0 = time.perf_counter()
    oracle.lanczos_csr(H, 1, 1e-300, nH, max_steps=steps)
    return time.perf_counter() - t0


def oracle_extrapolate(points, N):
    """Least-squares fit of t(s) = a s + b s^2 / 2 (SpMV plus reorthogonalisation against j vectors
    per step) to timed (steps, seconds) points; the time of an N-step run in ms."""
    A = np.array([[s, s * s / 2.0] for s, _ in points])
    (a, b), *_ = np.linalg.lstsq(A, np.array([t for _, t in points]), rcond=None)
    a, b = max(a, 0.0), max(b, 0.0)
    return (N * a + N * N * b / 2.0) * 1e3


# Oracle Lanczos steps of the timed sample runs per workload: two runs for the cpu_baseline leg
# (about 10-30 s of CPU work together on one core), one run per step of the reference arm.
ORACLE_SAMPLE_STEPS = {"c1": (10, 30), "c2": (10, 30), "c3": (2, 5)}
REF_STEP_STEPS = {"c1": (10, 30), "c2": (4, 12), "c3": (1, 3)}


def oracle_desc(cfg, N, what):
    _, _, full_s = golden_eigs(cfg)
    desc = dict(kind="oracle", cores=1, sample=(
        f"oracle Lanczos (FP64, full reorthogonalisation, 1 thread) on the same matrix: {what}; per-step cost "
        f"a + b j fitted, extrapolated to the {N} steps the full oracle run needs to reach Ritz residual 1e-12 ||H||"))
    if full_s is not None:
        desc["full_run_measured_s"] = full_s
        desc["full_run_note"] = (f"the full {N}-step oracle run that wrote the stored eigenvalues took {full_s:.0f} s on "
                                 f"one core of the x86 build host")
    return desc


def oracle_sample(cfg, layout, dev=None):
    """The oracle (plain single-threaded FP64 Lanczos, full reorthogonalisation) on a bounded
    sample of the same workload: two short runs of s1 < s2 Lanczos steps fix the per-step cost
    a + b j (SpMV plus reorthogonalisation against j vectors); the time to the converged step
    count N of the full oracle run (stored with the reference eigenvalues) is N a + N^2 b / 2.
    Returns (estimate ms, description)."""
    H, nH = oracle_matrix(cfg, layout, dev)
    _, N, _ = golden_eigs(cfg)
    N = N or 300
    s1, s2 = ORACLE_SAMPLE_STEPS.get(cfg, (10, 30))
    t = [oracle_run_s(H, nH, s) for s in (s1, s2)]
    desc = oracle_desc(cfg, N, f"{s1} and {s2} steps timed ({t[0]:.2f} s, {t[1]:.2f} s)")
    desc["sample_s"] = sum(t)
    return oracle_extrapolate([(s1, t[0]), (s2, t[1])], N), desc


def csb_sample(cfg, layout, nb, bytes_per_call, gpu_ms):
    """The paper's CPU organisation of the SpMM (threaded CSB: tile rows then tile columns, OpenMP
    dynamic scheduling, FP32 values; Section 4.4) on all host cores, on the bench's matrix at the
    same block width. Median of 10 calls after 2 warm-ups; algorithmic bytes as for the GPU kernel."""
    import baseline
    import synth

    r, c, v = (_np(a) for a in host_coo(cfg, layout))
    M = baseline.CsbMatrix(layout.n, r, c, v)
    X = np.random.default_rng(3).standard_normal((layout.n, nb))
    Y = np.empty_like(X)
    for _ in range(2):
        M.spmm(X, Y)
    t = []
    for _ in range(10):
        t0 = time.perf_counter()
        M.spmm(X, Y)
        t.append(time.perf_counter() - t0)
    M.close()
    ms = float(np.median(t)) * 1e3
    threads = baseline.max_threads()
    return {"kind": "threaded CPU CSB SpMM (row pass over tile rows, column pass over tile columns, "
                    "OpenMP dynamic schedule, FP32 values)", "threads": threads, "nb": nb,
            "ms": ms, "gbs": bytes_per_call / (ms * 1e-3) / 1e9, "gpu_ms": gpu_ms,
            "gpu_speedup": ms / gpu_ms if gpu_ms > 0 else None}


# Multi-level guesses tried by the ablation: (top level of the intermediate block, the relative
# residual its solve runs to). The tolerance is about the eq. 12 residual ||H_21 x|| / ||H|| that
# the block leaves on the generator's matrices (levels <= 6: 2.5e-5, <= 7: 9e-6, <= 8: 1.3e-6 on the
# n = 500,000 workload), so each guess is as good as eq. 12 allows for its block.
GUESS_ML = ((6, 2e-5), (7, 8e-6), (8, 1e-6))


def guess_ablation(M, k, nb, tol, X, layout, stream, args, torch, wl, ms_one, st_one, n_small):
    """Initial-guess ablation in the spirit of Table 2: the headline solve's one-level eq. 12 guess
    (levels {0, 1}) against the paper's multi-level scheme (Section 3.3.1): LOBPCG on the leading
    levels <= q, started from the eq. 12 guess of levels {0, 1}, its result zero-padded as the guess
    of the full solve. Every variant is timed end to end with CUDA events, the guess included."""
    import synth

    lv = synth.level_starts(layout)
    gold = golden_eigs(wl["cfg"])[0]
    n_inner = int(lv[2])
    out = {"one_level": {"guess": "eq. 12, levels {0, 1}", "n_small": n_small, "ms": ms_one,
                         "iterations": st_one["iterations"], "refine_iterations": st_one["refine_iterations"],
                         "guess_relres": st_one.get("guess_relres", [None])[0]},
           "multi_level": []}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [fn() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, res[-1]

    # eq. 13: the same guess corrected by one application of the block preconditioner
    ms13, (lam, _, st, rc) = timed(lambda: M.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_small,
                                                   guess_correct=True, X_out=X))
    out["eq13"] = {"guess": "eq. 13: eq. 12 of levels {0, 1} corrected by the block preconditioner",
                   "n_small": n_small, "ms": ms13, "iterations": st["iterations"],
                   "refine_iterations": st["refine_iterations"], "status": int(rc),
                   "guess_relres_eq12": st["guess_relres"][0], "guess_relres_eq13": st["guess_relres"][1],
                   "max_relres": max(st["residual"][:k]), "speedup": ms_one / ms13 if ms13 > 0 else None}
    if gold is not None:
        out["eq13"]["eig_err_vs_oracle"] = float((np.abs(lam - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
    for q, gtol in GUESS_ML:
        if q + 2 >= len(lv) - 1:
            continue
        n_outer = int(lv[q + 1])

        def solve_ml():
            return M.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_outer, n_small_inner=n_inner,
                           guess_tol=gtol, X_out=X)

        ms, (lam, _, st, rc) = timed(solve_ml)
        row = {"guess": f"LOBPCG on levels <= {q} from the eq. 12 guess of levels {{0, 1}}", "n_small": n_outer,
               "n_small_inner": n_inner, "guess_tol": gtol, "ms": ms, "iterations": st["iterations"],
               "refine_iterations": st["refine_iterations"], "status": int(rc),
               "max_relres": max(st["residual"][:k]), "speedup": ms_one / ms if ms > 0 else None}
        if gold is not None:
            row["eig_err_vs_oracle"] = float((np.abs(lam - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
        out["multi_level"].append(row)
    return out


def precond_ablation(lob, synth, layout, k, nb, tol, n_small, stream, args, torch, wl, ms_one, st_one):
    """Preconditioner ablation: Section 4.3's own choice, the diagonal 256 x 256 tiles with FOM
    steps on the tile store (precond_block = 256), against dense 32 x 32 blocks eigendecomposed
    at create with FOM in each block's eigenbasis -- whichever of the two the headline does not
    use. Same matrix, guess and tolerance; each solve timed end to end with CUDA events."""
    alt = 32 if wl["bp"] == 256 else 256
    r, c, v = synth.generate_device(layout)
    t0 = time.perf_counter()
    M = lob.Matrix(layout.n, r, c, v, precond_block=alt)
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t0) * 1e3
    del r, c, v
    X = torch.empty((layout.n, nb), dtype=torch.float64, device="cuda")

    def solve_t():
        return M.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_small, X_out=X)

    solve_t()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [solve_t() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    lam, _, st, rc = res[-1]
    head = {"b_p": wl["bp"], "ms": ms_one, "iterations": st_one["iterations"],
            "refine_iterations": st_one["refine_iterations"], "precond_ms": st_one["phase_ms"]["precond"]}
    other = {"b_p": alt, "ms": ms, "iterations": st["iterations"], "refine_iterations": st["refine_iterations"],
             "precond_ms": st["phase_ms"]["precond"], "create_ms": create_ms, "status": int(rc),
             "max_relres": max(st["residual"][:k])}
    gold = golden_eigs(wl["cfg"])[0]
    if gold is not None:
        other["eig_err_vs_oracle"] = float((np.abs(lam - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
    tiles, dense = (head, other) if wl["bp"] == 256 else (other, head)
    out = {"diagonal_tiles": tiles, "dense_blocks": dense, "headline": "diagonal_tiles" if wl["bp"] == 256 else
           "dense_blocks", "tiles_speedup_over_dense": dense["ms"] / tiles["ms"] if tiles["ms"] > 0 else None}
    M.close()
    return out


def replica_layout(cfg, rank):
    """Replicas only: rank r solves its own seeded instance of the workload (seed + r)."""
    import synth
    base = synth.CONFIGS[cfg]
    return synth.config_layout(cfg, seed=base["seed"] + rank)


def reduce_max(x, dist, device):
    """The slowest rank's time (every rank gets it); x unchanged without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def serving_requests(count, rate, seed=2024):
    """The serving workload: Poisson arrivals (mean `rate` per second), sizes log-uniform in
    [2,000, 200,000], k uniform in {1..8}, nb the next power of two >= k, ~30 nonzeros per row,
    levels interpolated from the size, one generator seed per request."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    n = np.exp(rng.uniform(np.log(2000), np.log(200000), count)).astype(np.int64)
    k = rng.integers(1, 9, count)
    nb = np.array([1 << int(np.ceil(np.log2(x))) for x in k])
    return [dict(t=float(t[i]), n=int(n[i]), k=int(k[i]), nb=int(nb[i]), seed=1000 + i) for i in range(count)]


def run_serving(args, lob, synth, torch):
    """Continuous-batching server (lob_server_*) on the serving workload, mixed precision,
    tol 1e-8 ||H||, block-Jacobi b_p = 32, eq. 12 guess; 60 GB admission budget. Matrices are
    built before the clock starts (resident in HBM). Reports p50/p99 latency (submit to done,
    queueing included) and solves/s, plus a closed batch of the first requests served mixed
    against the same requests solved one at a time by the plain FP64 solver."""
    reqs = serving_requests(args.serve_requests, args.serve_rate)
    t0 = time.perf_counter()
    for q in reqs:
        L = synth.layout(q["n"], synth.interp_levels(q["n"]), 30, q["seed"])
        r, c, v = synth.generate_device(L)
        q["M"] = lob.Matrix(q["n"], r, c, v, precond_block=32)
        q["n_small"] = int(synth.level_starts(L)[2])
        del r, c, v
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0

    def serve(sample, arrivals, mode="mixed", engine="lockstep"):
        srv = lob.Server(budget_bytes=60 << 30, max_active=args.serve_slots, engine=engine)
        ids = {}
        res = {}
        i = 0
        late = 0.0
        t_start = time.perf_counter()
        while len(res) < len(sample):
            now = time.perf_counter() - t_start
            while i < len(sample) and (not arrivals or sample[i]["t"] - sample[0]["t"] <= now):
                q = sample[i]
                rid = srv.submit(q["M"], q["k"], q["nb"], 1e-8, mode=mode, precond=True, n_small=q["n_small"])
                ids[rid] = i
                if arrivals:
                    late = max(late, now - (q["t"] - sample[0]["t"]))
                i += 1
            nd = srv.progress(wait=False)
            if nd:
                for rid in list(ids):
                    if rid in res:
                        continue
                    r = srv.poll(rid)
                    if r["state"] == lob.REQ_DONE:
                        res[rid] = r
        wall = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        out = [None] * len(sample)
        for rid, j in ids.items():
            out[j] = res[rid]
        return out, wall, st, late

    torch.cuda.nvtx.range_push("serve")  # marks the timed serving run for profilers
    out, wall, st, late = serve(reqs, True)
    torch.cuda.nvtx.range_pop()
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in out])
    ok = sum(1 for r in out if r["rc"] == lob.LOB_OK)
    failed = [dict(n=q["n"], k=q["k"], nb=q["nb"], rc=int(r["rc"]), iterations=int(r["stats"]["iterations"]))
              for q, r in zip(reqs, out) if r["rc"] != lob.LOB_OK]
    serving = {"workload": f"{len(reqs)} requests, Poisson {args.serve_rate:g}/s, n log-uniform [2000, 200000], "
                           f"k U{{1..8}}, nb = next pow2 >= k, ~30 nnz/row, mixed, tol 1e-8, b_p=32, budget 60 GB",
               "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "mean_ms": float(lat.mean()), "solves_per_s": len(out) / wall, "wall_s": wall, "converged": ok,
               "not_converged": failed[:20],
               "max_submit_lateness_ms": late * 1e3, "peak_bytes": int(st["bytes_peak"]),
               "spmm_products": int(st["spmm_products"]), "spmm_launches": int(st["spmm_launches"]),
               "rounds": int(st["rounds"]), "host_ms": st["host_ms"], "device_wait_ms": st["wait_ms"],
               "matrix_build_s": build_s}
    # closed batch: the first requests all at once, served mixed vs one at a time in FP64
    sample = reqs[:args.serve_compare]
    outb, wallb, stb, _ = serve(sample, False)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    lam64 = []
    for q in sample:
        lam, _, _, rc = q["M"].solve(q["k"], q["nb"], 1e-8, mode="fp64", precond=True, n_small=q["n_small"])
        lam64.append(lam)
    torch.cuda.synchronize()
    wall64 = time.perf_counter() - t1
    diff = max(float((np.abs(r["lam"] - l) / np.maximum(np.abs(l), 1.0)).max()) for r, l in zip(outb, lam64))
    serving["compare"] = {"requests": len(sample), "served_mixed_s": wallb, "single_fp64_s": wall64,
                          "served_mixed_solves_per_s": len(sample) / wallb,
                          "single_fp64_solves_per_s": len(sample) / wall64,
                          "speedup_served_mixed_over_single_fp64": wall64 / wallb,
                          "max_eig_rel_diff": diff, "spmm_products": int(stb["spmm_products"]),
                          "spmm_launches": int(stb["spmm_launches"])}
    for q in reqs:
        q["M"].close()
    return serving


def run_batched_small(args, lob, synth, torch):
    """The batched small-instance workload: 4,096 matrices, n uniform in [256, 4,096], ~40
    nonzeros per row, k = 4, nb = 8, tol 1e-8, random start, no preconditioner -- all solved by
    one persistent kernel schedule replayed from a CUDA graph (lob_batch_solve): an FP32 phase
    (FP32 values, X and products) then an FP64 phase, FP64 Cholesky factors and Rayleigh-Ritz
    solves throughout. The first call autotunes the schedule (slice height, threads per CTA,
    CTAs per SM) and is reported apart; the timed calls reuse its choice. Also: a sample solved
    one at a time by lob_solve (mixed) for the speedup, and in FP64 for the eigenvalue agreement;
    optionally the same batch on the lockstep serving engine."""
    rng = np.random.default_rng(4096)
    count = args.small_count
    ns = rng.integers(256, 4097, count)
    probs = []
    t0 = time.perf_counter()
    for i, n in enumerate(ns):
        L = synth.layout(int(n), synth.interp_levels(int(n)), 40, 50000 + i)
        r, c, v = synth.generate_device(L)
        probs.append((int(n), r, c, v))
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = lob.Batch(probs)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    kw = dict(mode="mixed", seed=1)
    lam, status, iters, _, st_tune = B.solve(4, 8, 1e-8, **kw)
    k0 = lob.kernel_launches()
    runs = []
    for _ in range(max(1, args.small_reps)):
        lam, status, iters, _, st = B.solve(4, 8, 1e-8, **kw)
        runs.append(st)
    launches = (lob.kernel_launches() - k0) // len(runs)
    kern = sorted(r["kernel_ms"] for r in runs)
    wall = sorted(r["wall_ms"] for r in runs)
    ok = int((status == lob.LOB_OK).sum())
    # the same instances one at a time through lob_solve
    samp = list(range(0, count, max(1, count // args.small_sample)))[:args.small_sample]
    mats = {i: lob.Matrix(*probs[i]) for i in samp}
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i in samp:
        mats[i].solve(4, 8, 1e-8, mode="mixed", precond=False, seed=1 + i, stats=False)
    torch.cuda.synchronize()
    seq = (time.perf_counter() - t1) / len(samp)
    diff = 0.0
    for i in samp:
        lam64, _, _, _ = mats[i].solve(4, 8, 1e-8, mode="fp64", precond=False, seed=1 + i, stats=False)
        diff = max(diff, float((np.abs(lam[i] - lam64) / np.maximum(np.abs(lam64), 1.0)).max()))
    for M in mats.values():
        M.close()
    out = {"workload": f"{count} matrices, n uniform [256, 4096], ~40 nnz/row, k=4, nb=8, tol 1e-8, "
                       f"no preconditioner; FP32 phase then FP64 phase, FP64 Rayleigh-Ritz",
           "schedule": "one persistent kernel (CTA per instance, atomic ticket, largest first) in a CUDA graph",
           "autotuned": {"tile": st_tune["tile"], "threads": st_tune["threads"], "per_sm": st_tune["per_sm"],
                         "candidates": st_tune["candidates"], "tune_ms": st_tune["tune_ms"]},
           "kernel_ms_median": kern[len(kern) // 2], "kernel_ms_min": kern[0],
           "wall_ms_median": wall[len(wall) // 2], "reps": len(runs),
           "instances_per_s": count / (wall[len(wall) // 2] / 1e3), "converged": ok,
           "iterations_mean": float(iters[:, 0].mean()), "iterations_max": int(iters[:, 0].max()),
           "fp64_phase_iterations_mean": float(iters[:, 1].mean()),
           "kernel_launches_per_call": int(launches), "rows": int(st["rows"]), "sell_entries": int(st["entries"]),
           "work_bytes": int(st["work_bytes"]), "generate_s": gen_s, "batch_build_s": build_s,
           "sequential_lob_solve_s_per_instance": seq,
           "speedup_batched_over_sequential": seq * count / (wall[len(wall) // 2] / 1e3),
           "max_eig_rel_diff_vs_fp64_single": diff, "sample": len(samp)}
    B.close()
    if args.small_lockstep:
        mats = [lob.Matrix(*p) for p in probs]
        srv = lob.Server(budget_bytes=60 << 30, max_active=count, engine="lockstep")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [srv.submit(M, 4, 8, 1e-8, mode="mixed", precond=False, seed=1 + i) for i, M in enumerate(mats)]
        done = set()
        while len(done) < count:
            if srv.progress(wait=True):
                for i in ids:
                    if i not in done and srv.poll(i)["state"] == lob.REQ_DONE:
                        done.add(i)
        torch.cuda.synchronize()
        out["lockstep_engine_wall_s"] = time.perf_counter() - t0
        srv.close()
        for M in mats:
            M.close()
    return out


def run_vblock(lob, torch, layout, n, rows, cols, vals, nb, reps=10):
    """The variable-size block store (levels cut into blocks of at most 256 rows, 8 + 8-bit
    offsets, 6 B per stored entry) and its FP32-value SpMM on the bench's matrix: median of
    `reps` launches (CUDA events, inputs larger than L2) after two warm-ups."""
    import synth
    groups = synth.level_starts(layout)[:-1]
    t0 = time.perf_counter()
    V = lob.VMatrix(n, rows, cols, vals, groups, 256)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    inf = V.info()
    X = torch.randn((n, nb), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    for _ in range(2):
        V.spmm(X, out=Y)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        V.spmm(X, out=Y)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    # algorithmic bytes: 6 B per stored entry, block tables, X read as FP32 and Y written in FP64
    alg = inf["nnz"] * 6 + inf["ntiles"] * 12 + (inf["nblocks"] + 1) * 16 + n * nb * (4 + 8)
    V.close()
    del X, Y
    torch.cuda.empty_cache()
    return {"store": "variable-size blocks (levels cut at 256 rows), (r << 8) | c + FP32 value",
            "nblocks": int(inf["nblocks"]), "blocks_stored": int(inf["ntiles"]), "store_bytes": int(inf["store_bytes"]),
            "bytes_per_entry": inf["store_bytes"] / inf["nnz"], "build_ms": build_ms, "ms": ms,
            "algorithmic_bytes": alg, "gbs": alg / (ms * 1e-3) / 1e9, "kernel": "k_vspmm (one CTA per block row)"}


def run_kernels(args, lob, M, info, torch, make_matrix):
    """Each hot-path kernel alone at the workload's sizes (CUDA events, L2 flushed between
    repetitions): the symmetric SpMM in its three arithmetics, the 48 x 48 double-float Gram,
    the n x 48 by 48 x 16 double-float linear combination, the 48 x 48 Rayleigh-Ritz solve and the
    preconditioner on dense 32 x 32 blocks and on the diagonal tiles.
    Prints one JSON line; a clean target for profiler captures of one launch of each kernel."""
    n, nb = M.n, 16
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn((n, nb), dtype=torch.float64, device="cuda", generator=g)
    S = torch.randn((n, 48), dtype=torch.float64, device="cuda", generator=g)
    T = torch.randn((n, 48), dtype=torch.float64, device="cuda", generator=g)
    Cm = torch.randn((48, 16), dtype=torch.float64, device="cuda", generator=g)
    Gd = S[:4096].T @ T[:4096]
    Gs = (Gd + Gd.T) / 2
    Ms = S[:4096].T @ S[:4096]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}

    def timeit(name, fn, reps=10, **extra):
        for _ in range(2):
            fn()
        ms = []
        for _ in range(reps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[name] = dict(ms=float(np.median(ms)), **extra)

    nnz, ntiles, nt = int(info["nnz"]), int(info["ntiles"]), (n + 255) // 256
    for mode, sv in (("mixed", 4), ("df64", 8), ("fp64", 8)):
        byts = nnz * (sv + 4) + ntiles * 12 + (nt + 1) * 8 + n * nb * (8 + 8)
        timeit("spmm_" + mode, lambda mode=mode: M.spmm(X, mode), algorithmic_bytes=byts)
    timeit("gram_df_48x48", lambda: lob.gram(S, T, "df64"), df_macs=n * 48 * 48, algorithmic_bytes=n * 96 * 8)
    timeit("gram_tc_48x48", lambda: lob.gram(S, T, "mixed"), algorithmic_bytes=n * 96 * 8)
    timeit("lincomb_df_48x16", lambda: lob.lincomb(S, Cm, "df64"), df_macs=n * 48 * 16,
           algorithmic_bytes=n * (48 + 16) * 8)
    timeit("lincomb_tc_48x16", lambda: lob.lincomb(S, Cm, "mixed"), algorithmic_bytes=n * (48 + 16) * 8)
    C48 = torch.randn((48, 48), dtype=torch.float64, device="cuda", generator=g)
    timeit("lincomb_tc_48x48", lambda: lob.lincomb(S, C48, "mixed"), algorithmic_bytes=n * (48 + 48) * 8)
    timeit("rayleigh_ritz_df_48", lambda: lob.rayleigh_ritz(Gs, Ms, "mixed"), reps=20)
    mu = torch.linspace(-5.0, -4.0, nb, dtype=torch.float64, device="cuda")
    # the preconditioner both ways: dense 32 x 32 blocks (eigenbasis FOM) and the diagonal tiles
    for bp in (32, 256):
        Mp = M if int(info.get("precond_block", 0)) == bp else make_matrix(bp)
        if bp == 256:  # R and W; the diagonal tiles come from the tile store (counted with the SpMM)
            timeit("precond_tiles_fom3", lambda Mp=Mp: Mp.precond_apply(mu, X, solve="fom", steps=3),
                   algorithmic_bytes=2 * n * nb * 8)
        else:
            timeit("precond_fom3", lambda Mp=Mp: Mp.precond_apply(mu, X, solve="fom", steps=3),
                   algorithmic_bytes=((n + bp - 1) // bp) * bp * bp * 4 + 2 * n * nb * 8)
        if Mp is not M:
            Mp.close()
    for v in out.values():
        if "algorithmic_bytes" in v:
            v["gbs"] = v["algorithmic_bytes"] / (v["ms"] * 1e-3) / 1e9
        if "df_macs" in v:  # 12 FP32 instructions per double-float multiply-add
            v["fp32_tinst_s"] = 12 * v["df_macs"] / (v["ms"] * 1e-3) / 1e12
    print(json.dumps({"kernels": out, "n": n, "nnz_stored": nnz}))


def run_reference(args, wl):
    """The reference arm: the oracle as it stands on one host core. Each step is one bounded
    oracle Lanczos call on the workload's matrix, alternating two lengths; ms_per_step is the
    measured time of those calls, and value is the full oracle solve extrapolated from all timed
    steps (per-step cost a + b j) to the step count of the stored reference run."""
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    layout = synth.config_layout(wl["cfg"])
    dev = None
    try:  # input generation only: the device generator is much faster than the host's at 1.2e9 entries
        import torch
        if torch.cuda.is_available():
            dev = synth.generate_device(layout)
    except Exception:
        dev = None
    H, nH = oracle_matrix(wl["cfg"], layout, dev)
    del dev
    _, N, _ = golden_eigs(wl["cfg"])
    N = N or 300
    lens = REF_STEP_STEPS.get(wl["cfg"], (10, 30))
    points = []
    for i in range(args.warmup + args.steps):
        s = lens[i % 2]
        t = oracle_run_s(H, nH, s)
        if i >= args.warmup:
            points.append((s, t))
    if len({s for s, _ in points}) < 2:  # one timed length cannot fix two coefficients
        points.append((lens[1 - lens.index(points[0][0])], oracle_run_s(H, nH, lens[1 - lens.index(points[0][0])])))
    v = oracle_extrapolate(points, N)
    step_ms = float(np.mean([t for _, t in points[:args.steps]])) * 1e3
    desc = oracle_desc(wl["cfg"], N, f"each step one call of {lens[0]} or {lens[1]} steps, alternating")
    line = {"impl": "reference", "metric": "time-to-k-eigenpairs", "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "n": int(layout.n)},
            "value_note": "value = the full oracle solve extrapolated from the timed steps; ms_per_step = their "
                          "measured mean",
            "cpu_baseline": dict(desc, value=v, unit="ms"),
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-csb", action="store_true", help="skip the threaded CPU CSB SpMM baseline")
    ap.add_argument("--no-ablation", action="store_true", help="skip the multi-level initial-guess ablation")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-lanczos", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-compare", type=int, default=100)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-vblock", action="store_true", help="skip the variable-size block store's SpMM")
    ap.add_argument("--small-count", type=int, default=4096)
    ap.add_argument("--small-sample", type=int, default=64)
    ap.add_argument("--small-reps", type=int, default=3)
    ap.add_argument("--small-lockstep", action="store_true", help="also run the batch on the lockstep engine")
    ap.add_argument("--kernels", action="store_true", help="time each hot-path kernel alone and exit")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch

    import paper_1609_01689_gb300 as lob
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- setup (not timed): generate on the device, build the tile store and preconditioner
    layout = replica_layout(wl["cfg"], rank)
    n = int(layout.n)
    rows, cols, vals = synth.generate_device(layout)
    t0 = time.perf_counter()
    M = lob.Matrix(n, rows, cols, vals, precond_block=wl["bp"])
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t0) * 1e3
    info = M.info()
    if args.kernels:
        return run_kernels(args, lob, M, info, torch,
                           lambda bp: lob.Matrix(n, rows, cols, vals, precond_block=bp))
    # the host legs (end to end from pinned host buffers, the oracle sample, the threaded CPU SpMM)
    # use one pinned host copy of the COO; the device copy is then released
    if not args.no_e2e or (rank == 0 and not (args.no_cpu and args.no_csb)):
        host_coo(wl["cfg"], layout, dev=(rows, cols, vals))
    vblock = None
    if rank == 0 and not args.no_vblock:
        vblock = run_vblock(lob, torch, layout, n, rows, cols, vals, wl["nb"])
    del rows, cols, vals
    torch.cuda.empty_cache()
    n_small = int(synth.level_starts(layout)[2])
    k, nb, tol = wl["k"], wl["nb"], wl["tol"]
    X = torch.empty((n, nb), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def solve(mode):
        return M.solve(k, nb, tol, mode=mode, precond=True, n_small=n_small, X_out=X)

    for _ in range(args.warmup):
        solve("mixed")
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = lob.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    stats = []
    lam = None
    for _ in range(args.steps):
        lam, _, st, rc = solve("mixed")
        stats.append((st, rc))
    ev1.record(stream)
    barrier()
    launches = lob.kernel_launches() - launches0
    clocks = sampler.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = reduce_max(ms_total, dist, "cuda")
    ms_step = ms_total / args.steps

    # SpMM roofline (the mixed-precision SpMM, the solve's dominant product): algorithmic bytes /
    # launch time (CUDA events on the solver's stream) over the timed solves
    spmm_bytes = sum(s["spmm_by_mode"]["mixed"]["bytes"] for s, _ in stats)
    spmm_ms = sum(s["spmm_by_mode"]["mixed"]["ms"] for s, _ in stats)
    spmm_calls = sum(s["spmm_by_mode"]["mixed"]["calls"] for s, _ in stats)
    peak, peak_src = read_peaks()
    achieved = spmm_bytes / (spmm_ms * 1e-3) / 1e9 if spmm_ms > 0 else 0.0

    out = {"metric": "time-to-k-eigenpairs", "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None,
           "dtype": "mixed: f32-value SpMM with f64 sums; f64-class Gram and X*C (double-float, or bf16-digit "
                    "splits on the tensor cores); f64 Cholesky-QR factors and Rayleigh-Ritz; f64-value refinement SpMM",
           "data": "synthetic",
           "config": {"workload": wl["name"], "n": n, "nnz_stored": int(info["nnz"]), "ntiles": int(info["ntiles"]),
                      "k": k, "nb": nb, "b_p": wl["bp"], "tol": tol, "mode": "mixed+fp64 refinement",
                      "l2": "inputs larger than L2 (tile store %.2f GB)" % (info["store_bytes"] / 1e9),
                      "parallelism": f"replicas x{world}"},
           "roofline": {"bound": "hbm", "kernel": "symmetric SpMM (mixed)", "achieved": achieved, "peak": peak,
                        "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                        "traffic": SPMM_TRAFFIC.get(wl["cfg"]),
                        "launches": spmm_calls, "avg_launch_ms": spmm_ms / max(spmm_calls, 1),
                        "bytes_per_launch": spmm_bytes / max(spmm_calls, 1)},
           "clocks": clocks, "gpu_launches": launches}
    # the FP64-value refinement product: bound by the FP64 pipe, so its fraction is of FP64 flops
    f64_ms = sum(s["spmm_by_mode"]["fp64"]["ms"] for s, _ in stats)
    f64_calls = sum(s["spmm_by_mode"]["fp64"]["calls"] for s, _ in stats)
    if f64_calls:
        flops = 4.0 * nb * info["nnz"] - 2.0 * nb * n  # 4 nb per stored off-diagonal entry, 2 nb per diagonal
        ach = f64_calls * flops / (f64_ms * 1e-3)
        out["roofline_fp64_spmm"] = {"bound": "alu", "pipe": "fp64", "kernel": "symmetric SpMM (FP64 values)",
                                     "achieved": ach / 1e12, "peak": FP64_NOMINAL_FLOPS / 1e12, "unit": "TFLOP/s",
                                     "frac": ach / FP64_NOMINAL_FLOPS, "peak_source": "nominal",
                                     "launches": f64_calls, "avg_launch_ms": f64_ms / f64_calls}
    st0 = stats[-1][0]
    if rank == 0 and not args.no_ablation and wl["cfg"] != "c3":
        out["precond_ablation"] = precond_ablation(lob, synth, layout, k, nb, tol, n_small, stream, args, torch,
                                                   wl, ms_step, st0)
    if rank == 0 and not args.no_ablation:
        out["guess_ablation"] = guess_ablation(M, k, nb, tol, X, layout, stream, args, torch, wl, ms_step, st0,
                                               n_small)
    out["solve"] = {"iterations": st0["iterations"], "refine_iterations": st0["refine_iterations"],
                    "status": int(stats[-1][1]), "phase_ms": st0["phase_ms"], "create_ms": create_ms,
                    "spmm_by_mode": st0["spmm_by_mode"], "max_relres": max(st0["residual"][:k])}
    gold = golden_eigs(wl["cfg"])[0]
    if gold is not None and rank == 0 and lam is not None:
        err = np.abs(lam - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)
        out["eig_err_vs_oracle"] = float(err.max())

    # ---- plain FP64 solver on the same workload (not in the timed region)
    if not args.no_fp64:
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam64, _, st64, rc64 = solve("fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        fp = {"ms": t64, "iterations": st64["iterations"], "status": int(rc64),
              "speedup_mixed_over_fp64": t64 / ms_step}
        if gold is not None:
            fp["eig_err_vs_oracle"] = float((np.abs(lam64 - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
        out["fp64_solver"] = fp

    # ---- the same mixed solve with its double-float options: Cholesky-QR factors and Rayleigh-Ritz
    # in double-float, and double-float values and products in the refinement SpMM
    if not args.no_fp64:
        kw = dict(rr_arith="df", refine_arith="df")
        M.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_small, X_out=X, **kw)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam_d, _, st_d, rc_d = M.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_small, X_out=X, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        dfv = {"ms": e0.elapsed_time(e1), "iterations": st_d["iterations"],
               "refine_iterations": st_d["refine_iterations"], "status": int(rc_d),
               "rr_ms": st_d["phase_ms"]["rr"], "spmm_ms": st_d["phase_ms"]["spmm"],
               "what": "double-float Cholesky-QR factors and Rayleigh-Ritz, double-float-value refinement SpMM"}
        if gold is not None:
            dfv["eig_err_vs_oracle"] = float((np.abs(lam_d - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
        out["mixed_df_variant"] = dfv

    # ---- the Lanczos baseline (single vector, full reorthogonalisation, FP64) to the same residual
    if not args.no_lanczos:
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam_l, _, st_l, rc_l = lob.lanczos(M, k, tol, max_steps=1200, vectors=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_l = e0.elapsed_time(e1)
        la = {"ms": t_l, "steps": st_l["steps"], "status": int(rc_l), "spmv_ms": st_l["spmv_ms"],
              "basis_bytes": st_l["device_bytes"], "speedup_mixed_lobpcg_over_lanczos": t_l / ms_step}
        if lam is not None:
            la["max_eig_rel_diff_vs_lobpcg"] = float((np.abs(lam_l - lam) / np.maximum(np.abs(lam), 1.0)).max())
        if gold is not None:
            la["eig_err_vs_oracle"] = float((np.abs(lam_l - gold[:k]) / np.maximum(np.abs(gold[:k]), 1.0)).max())
        out["lanczos_baseline"] = la

    # ---- end to end through the public API from pinned host buffers
    if not args.no_e2e:
        hr, hc, hv = host_coo(wl["cfg"], layout)
        Xh = torch.empty((n, nb), dtype=torch.float64).pin_memory()
        steps_e2e = max(1, min(2, args.steps))
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            Me = lob.Matrix(n, hr.numpy(), hc.numpy(), hv.numpy(), precond_block=wl["bp"])
            lam_e, Xd, _, _ = Me.solve(k, nb, tol, mode="mixed", precond=True, n_small=n_small)
            Xh.copy_(Xd)
            torch.cuda.synchronize()
            Me.close()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / steps_e2e
        out["e2e"] = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(hr.numel() * 24),
                      "d2h_bytes_per_step": int(n * nb * 8 + k * 8),
                      "includes": "H2D of the COO, tile build + preconditioner setup, solve, D2H of X and lambda"}

    if vblock is not None:
        peak_v, _ = read_peaks()
        vblock["frac_of_hbm"] = vblock["gbs"] / peak_v
        vblock["fixed_tile_kernel_ms"] = spmm_ms / max(spmm_calls, 1)
        out["vblock_spmm"] = vblock
    if rank == 0 and not args.no_serve:
        out["serving"] = run_serving(args, lob, synth, torch)
    if rank == 0 and not args.no_small:
        out["batched_small"] = run_batched_small(args, lob, synth, torch)

    if rank == 0 and not args.no_cpu:
        ms_cpu, desc = oracle_sample(wl["cfg"], layout)
        out["cpu_baseline"] = dict(desc, value=ms_cpu, unit="ms")
    if rank == 0 and not args.no_csb and spmm_calls > 0:
        out["cpu_csb_spmm"] = csb_sample(wl["cfg"], layout, nb, spmm_bytes / spmm_calls, spmm_ms / spmm_calls)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
