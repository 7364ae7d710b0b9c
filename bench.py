#!/usr/bin/env python
"""Benchmark of the GB300 three-body eigensolver (arXiv 2111.02534 hot path).

One step = one tps_solve of the 1D workload with n = 512 points per Jacobi coordinate
(M/m = 40, v0 tuned to a heavy-light binding of 1e-3, 8 lowest heavy-exchange-even
eigenpairs, block size 8, FP64): every row of the hot path runs inside it (H-apply,
preconditioner, projectors, GMRES, block orthogonalisation, Rayleigh-Ritz, restarts).

metric  eigenpairs/sec counting only pairs whose eigenvalue is within 1e-10 relative of
        the oracle's (tests/golden/evals_1d_n512.json, written by oracle-only code);
        the H-apply / mode-product throughput is reported in ``roofline``.
Multi-GPU: replicas only (one independent solve per rank, no collective on the data
path); value = pairs of all ranks / max-over-ranks time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import threading
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigenpairs/sec at rel. eigenvalue err ≤1e-10; H-apply TFLOP/s vs peak"
UNIT = "eigenpairs/s"
WORKLOAD = "1d_n512"
REL_TOL = 1e-10
# FP64 FMA peak: 2 FP64 FMA units' worth of work per SM per clock (4 flop/clk/SM, the
# nominal 1.25 TFLOP/s of GB300 at 152 SMs x 2070 MHz; a throughput probe reached 95 %)
FP64_FLOP_PER_CLK_PER_SM = 4
N_SM = 152
SM_MAX_MHZ = 2070.0
# digit-pair products of the tensor-core FP64 emulation (9 wave-function digits, 10
# mode-matrix digits, levels i + j <= 9 kept): each one a BF16 MMA over the full product
TC_PAIRS = 54
# DRAM bytes (read + write) per launch of each kernel, mean over the launches of one ncu
# capture of the kernel on this workload; a kernel that changes after its capture is
# removed from this table
TRAFFIC_BYTES_PER_LAUNCH = {"k_tf32_gemm": 5.08e6}
# the same for kernels whose launches cover a varying number of vectors: (bytes per launch,
# bytes per vector), fitted to two captured launches of different width (k_oz_gemm: 6 and 4
# vectors, 49.65 and 35.66 MB)
TRAFFIC_AFFINE = {"k_oz_gemm": (7.68e6, 6.99e6)}
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense tensor rates per GPU (TF32, BF16)
# BF16 digit-pair products per FP64 multiply-add of the split block update
SPLIT_UPDATE_PAIRS = 34


def traffic_per_launch(name, kd):
    """DRAM bytes per launch of a kernel from its ncu capture (None if not captured since
    its last change); for kernels over a varying vector count, at the bench's mean count."""
    if name in TRAFFIC_AFFINE and kd.get("vectors_per_launch"):
        a, b = TRAFFIC_AFFINE[name]
        return a + b * kd["vectors_per_launch"]
    return TRAFFIC_BYTES_PER_LAUNCH.get(name)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-streams", type=int, default=32)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def aggregate(local_seconds, local_pairs, world, device=None):
    """Max time over ranks and total passing pairs (all-reduce when world > 1)."""
    if world == 1:
        return local_seconds, local_pairs
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    p = torch.tensor([float(local_pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(p.item()))


def golden():
    with open(os.path.join(ROOT, "tests", "golden", f"evals_{WORKLOAD}.json")) as f:
        return json.load(f)


def passing_pairs(lam, ref):
    lam = np.asarray(lam)
    n = min(len(lam), len(ref))
    ref = np.asarray(ref)[:n]
    # error relative to |lambda_i|, floored at the ground-state binding energy |lambda_0|:
    # an excited level that happens to sit next to zero has no meaningful relative error
    scale = np.maximum(np.abs(ref), np.abs(ref[0])) if n else ref
    rel = np.abs(lam[:n] - ref) / scale
    return int(np.sum(rel <= REL_TOL)), float(rel.max()) if n else float("inf")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        # the timed region starts once nvidia-smi has initialised and taken its first
        # sample, so that its start-up does not fall inside it
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.reader.join(timeout=5)
        self.out = "".join(self.lines)

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 7]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(w, v0):
    """The oracle as it stands on this host: LOBPCG for the lowest eigenpair of the same
    workload (a bounded sample of the 8-pair solve).  Returns (pairs/s, seconds, cores)."""
    from oracle.hamiltonian import problem_1d
    from oracle.eig import lowest_iterative
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, v0, w.sigma)
    t0 = time.perf_counter()
    lam, _ = lowest_iterative(P, 1, 1, tol=1e-12, extra=2)
    dt = time.perf_counter() - t0
    ref = golden()["evals"][0]
    ok = abs(lam[0] - ref) / abs(ref) <= REL_TOL
    return (1.0 if ok else 0.0) / dt, dt, os.cpu_count()


def blas_threads():
    """Threads of NumPy's BLAS (threadpoolctl when installed, else the environment's
    OMP/OPENBLAS setting, else None: the library default, one per core)."""
    try:
        from threadpoolctl import threadpool_info
        info = [d for d in threadpool_info() if d.get("user_api") == "blas"]
        if info:
            return {"library": info[0].get("internal_api"), "threads": info[0].get("num_threads")}
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return {"library": None, "threads": int(os.environ[var])}
    return None


def cpu_oracle_legs(w, v0):
    """The other CPU legs of the measurement, each the oracle as it stands:
    the NumPy tensor-form H-apply (Kronecker identity, two dense 512 x 512 mode products
    per vector) on the full n = 512 grid, and the dense LAPACK eigh of the x-even H of the
    n = 64 workload (2112 x 2112) that the GPU smoke test solves."""
    from oracle.hamiltonian import problem_1d
    from oracle.eig import lowest_dense
    from paper_2111_02534_gb300.inputs import WORKLOADS, random_block
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, v0, w.sigma)
    psi = random_block(8, P.N, 0)
    P.apply_kron(psi[:1])
    t0 = time.perf_counter()
    P.apply_kron(psi)
    dt_apply = (time.perf_counter() - t0) / 8
    flops = 2.0 * P.N * sum(w.n) + 3.0 * P.N
    w1 = WORKLOADS["1d_n64"]
    P1 = problem_1d(w1.M, w1.m, w1.hbar, w1.n, w1.L, w1.v0, w1.sigma)
    t0 = time.perf_counter()
    lowest_dense(P1, w1.k, 1)
    dt_eigh = time.perf_counter() - t0
    return {"apply_h_ms_per_vector": 1000.0 * dt_apply,
            "apply_h_gflops": flops / dt_apply / 1e9,
            "apply_h_what": "oracle tensor-form H-apply (NumPy FP64 matmul) on the full "
                            "512 x 512 grid, mean over 8 vectors",
            "dense_eigh_1d_n64_s": dt_eigh,
            "dense_eigh_1d_n64_pairs_per_s": w1.k / dt_eigh,
            "dense_eigh_what": "oracle dense LAPACK eigh of the x-even H of the n = 64 "
                               "workload (2112 x 2112, H assembled explicitly), 4 pairs"}


def run_sweep(tps, torch, nstreams, graph=0):
    """The 256-instance sweep (inputs.sweep_instances): contexts set up first (untimed: one
    full warm-up solve per grid size, one outer iteration per instance for its operators and
    workspace), then one timed tps_solve_batch over all of them.
    Pairs count when within 1e-10 of the oracle's eigenvalues (tests/golden/evals_sweep.json)."""
    path = os.path.join(ROOT, "tests", "golden", "evals_sweep.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)["instances"]
    ctxs, evecs = [], []
    for inst in gold:
        c = tps.Context(1, torch.cuda.current_device())
        c.set_masses(inst["M"], inst["m"], 1.0)
        c.set_grid([inst["n"], inst["n"]], [inst["L"], inst["L"]])
        mu = inst["M"] * inst["m"] / (inst["M"] + inst["m"])
        c.set_pair_potential(tps.GAUSS, tps.two_body_v0(1, mu, 1.0, inst["E0"], tps.GAUSS,
                                                        inst["sigma"], inst["n"], inst["L"]),
                             inst["sigma"])
        ctxs.append(c)
        evecs.append(torch.empty(4, c.info()[0], dtype=torch.float64, device="cuda"))
    seen = {}
    for i, inst in enumerate(gold):
        seen.setdefault(inst["n"], i)
    warm = sorted(seen.values())
    tps.solve_batch([ctxs[i] for i in warm], [4] * len(warm), tps.X_EVEN, 1e-12, 4,
                    [evecs[i] for i in warm], nstreams=nstreams)
    # set-up of every instance outside the timed region: one outer iteration per context
    # builds its parity-sector operator and allocates its solver workspace
    setup = tps.default_opts()
    setup.max_outer = 1
    setup.graph = graph
    tps.solve_batch(ctxs, [4] * len(ctxs), tps.X_EVEN, 1e-12, 4, evecs, opts=setup,
                    nstreams=nstreams)
    opts = tps.default_opts()
    opts.graph = graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, stats, status = tps.solve_batch(ctxs, [4] * len(ctxs), tps.X_EVEN, 1e-12, 4, evecs,
                                         opts=opts, nstreams=nstreams)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    passing, worst, misses = 0, 0.0, []
    for i, (l, g) in enumerate(zip(lam, gold)):
        ref = np.array(g["evals"])
        p, r = passing_pairs(l, ref)
        passing += p
        worst = max(worst, r)
        if p < len(ref):
            misses.append({"instance": i, "n": g["n"], "ref": g["evals"], "got": list(map(float, l)),
                           "rel_err": r})
    for c in ctxs:
        c.close()
    return {"instances": len(gold), "pairs_passing": passing, "eigenpairs_per_s": passing / dt,
            "wall_s": dt, "nstreams": nstreams, "host_threads": nstreams,
            "executor": "graph-captured outer loop per instance" if graph else
                        "host-driven outer loop per instance",
            "eigen_rel_err_max": worst, "misses": misses[:8],
            "workload": "256 instances, M/m~U[1,40], E0~logU[1e-4,1], sigma in {0.5,1,2}, "
                        "n in {128,192,256,384}, L=20, 4 x-even pairs each, block 4"}


def run_apply_2d(tps, torch, nvec=8, reps=5):
    """H-apply throughput on the 2D workload (n = 48 per Cartesian component, 5.3 M
    unknowns, 8 vectors): FP64 (FMA pipe and tensor-core emulation) and FP32 mode products,
    algorithmic 2N(4n)+3N flops per vector, CUDA events on the current stream; then the
    workload's solve (4 lowest pairs, block 8, all states), eigenpairs/s over solves whose
    pairs carry the solver's own residual certificate |lambda - theta| <= ||r|| <= 1e-10
    |theta| (no oracle eigenvalues exist at this size)."""
    from paper_2111_02534_gb300.inputs import WORKLOADS, random_normal_block
    w = WORKLOADS["2d_n48"]
    ctx = tps.Context(2, torch.cuda.current_device())
    ctx.set_masses(w.M, w.m, w.hbar)
    ctx.set_grid(list(w.n), list(w.L))
    ctx.set_pair_potential(tps.GAUSS, w.v0, w.sigma)
    N = ctx.info()[0]
    x = torch.from_numpy(random_normal_block(nvec, N, 5)).cuda()
    y = torch.empty_like(x)
    flops = nvec * (2.0 * N * sum(w.n) + 3.0 * N)
    out = {"workload": "2d_n48: M/m = 20, n = 48^4 (5,308,416 unknowns), 8 vectors",
           "nvec": nvec}
    for name, dt in (("fp64", tps.F64), ("fp64_tc", tps.F64_TC), ("fp32", tps.F32)):
        ctx.apply_h(x, y, 0.0, dtype=dt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.apply_h(x, y, 0.0, dtype=dt)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name + "_ms"] = ms
        out[name + "_tflops"] = flops / (ms / 1000.0) / 1e12
    del x, y
    # the 2D workload's solve
    ev = torch.empty(w.k, N, dtype=torch.float64, device="cuda")
    opts = tps.default_opts()
    opts.timing = 1
    lam, st = ctx.solve(w.k, tps.ANY, 1e-12, w.block, ev, opts=opts)   # warm-up (set-up)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, certified = [], 0
    hnorm = ctx.info()[1]
    for _ in range(2):
        e0.record()
        lam, st = ctx.solve(w.k, tps.ANY, 1e-12, w.block, ev, opts=opts)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1000.0)
        r = np.array(st.resid[:w.k]) * hnorm
        certified += int(np.sum(r <= 1e-10 * np.abs(np.asarray(lam))))
    out["solve"] = {"workload": "2d_n48: 4 lowest pairs, block 8, all states, tol 1e-12 ||H||",
                    "eigenpairs_per_s": certified / sum(times), "s_per_solve": sum(times) / 2,
                    "pairs_certified": certified, "pairs": 2 * w.k,
                    "eigenvalues": [float(v) for v in lam],
                    "outer_iters": st.outer_iters, "h_applies": st.h_applies,
                    "h_ms": st.h_ms, "prec_ms": st.prec_ms,
                    "certificate": "solver residual ||H x - theta x|| (fresh FP64 H-apply) <= "
                                   "1e-10 |theta| (Weyl bound); no oracle eigenvalues at 48^4"}
    ctx.close()
    return out


def workload_config(w, world):
    """The workload both arms report: the n = 512 1D problem and what is solved on it."""
    return {"workload": f"{WORKLOAD}: 1D heavy-heavy-light, M/m=40, n=512 per Jacobi coordinate "
                        "on [-20,20), v0 tuned to E0=1e-3, sigma=1, 8 lowest x-even eigenpairs, "
                        "block 8, tol 1e-12*||H||, eigenvalues within 1e-10 of the oracle",
            "parallelism": f"replicas x{world}", "l2": "flushed between timed steps",
            "unknowns": w.n[0] * w.n[1], "sector_unknowns": (w.n[0] // 2 + 1) * w.n[1]}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2111_02534_gb300.inputs import WORKLOADS
    w = WORKLOADS[WORKLOAD]
    v0 = golden()["v0"]
    for _ in range(args.warmup):
        cpu_oracle_sample(w, v0)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, cores = cpu_oracle_sample(w, v0)
        vals.append(v)
        secs.append(dt)
    total = sum(secs)
    value = args.steps / total if all(x > 0 for x in vals) else 0.0
    sample = ("oracle (NumPy/SciPy FP64, LOBPCG on the explicit Kronecker sum) computing the "
              "lowest x-even eigenpair of the n=512 workload per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(w, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl ours")
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    from paper_2111_02534_gb300 import tps
    from paper_2111_02534_gb300.inputs import WORKLOADS, random_normal_block

    w = WORKLOADS[WORKLOAD]
    gold = golden()
    ref = np.array(gold["evals"])
    mu_hl = w.M * w.m / (w.M + w.m)
    torch.cuda.synchronize()
    t_set0 = time.perf_counter()
    v0 = tps.two_body_v0(1, mu_hl, w.hbar, w.E0, tps.GAUSS, w.sigma, w.n[1], w.L[1])
    t_set1 = time.perf_counter()
    ctx = tps.Context(1, local)
    ctx.set_masses(w.M, w.m, w.hbar)
    ctx.set_grid(list(w.n), list(w.L))
    torch.cuda.synchronize()
    t_set2 = time.perf_counter()
    ctx.set_pair_potential(tps.GAUSS, v0, w.sigma)
    torch.cuda.synchronize()
    t_set3 = time.perf_counter()
    N, hnorm = ctx.info()
    stream = torch.cuda.current_stream()
    x0 = torch.from_numpy(random_normal_block(w.block, N, seed=1000 + rank)).cuda()
    evecs = torch.empty(w.k, N, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    opts = tps.default_opts()
    opts.timing = 1

    def step(o=opts):
        lam, st = ctx.solve(w.k, tps.X_EVEN, 1e-12, w.block, evecs, x0=x0, opts=o,
                            stream=stream)
        return lam, st

    t_first0 = time.perf_counter()
    step()          # the first solve also builds the sector operator and the workspace
    torch.cuda.synchronize()
    t_first1 = time.perf_counter()
    for _ in range(max(3, args.warmup) - 1):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    times, stats, pairs, rel_max = [], [], 0, 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)                      # L2 flushed between timed steps
            torch.cuda.synchronize()
            ev0.record(stream)
            lam, st = step()
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1000.0)
            stats.append(st)
            p, r = passing_pairs(lam, ref)
            pairs += p
            rel_max = max(rel_max, r)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    local_t = sum(times)
    T, total_pairs = aggregate(local_t, pairs, world, device="cuda")
    value = total_pairs / T

    # median of at least 10 solves (the timed steps plus extra untimed-for-value ones)
    med_times = list(times)
    while len(med_times) < 10:
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        med_times.append(ev0.elapsed_time(ev1) / 1000.0)
    setup = {"two_body_v0_ms": 1000.0 * (t_set1 - t_set0),
             "context_masses_grid_ms": 1000.0 * (t_set2 - t_set1),
             "pair_potential_ms": 1000.0 * (t_set3 - t_set2),
             "first_solve_ms": 1000.0 * (t_first1 - t_first0),
             "note": "host wall clock with device synchronisation; the first solve builds the "
                     "parity-sector operator, its tensor-core digit slices and TF32 eigenbases, "
                     "and the solver workspace, which later solves reuse"}
    solve_stats = {"solves": len(med_times), "median_ms": 1000.0 * statistics.median(med_times),
                   "mean_ms": 1000.0 * statistics.mean(med_times),
                   "min_ms": 1000.0 * min(med_times), "max_ms": 1000.0 * max(med_times),
                   "median_eigenpairs_per_s": len(ref) / statistics.median(med_times)}

    # end to end through the public API with host buffers: every step sets the potential
    # (the library evaluates it and uploads N doubles), copies the start block from pinned
    # host memory, solves, and reads eigenvectors and eigenvalues back to the host
    x0_host = x0.cpu().pin_memory()
    x0_dev = torch.empty_like(x0)
    evecs_host = torch.empty(w.k, N, dtype=torch.float64).pin_memory()
    e2e_t, e2e_pairs = 0.0, 0
    n_e2e = max(1, min(args.e2e_steps, args.steps))
    for _ in range(n_e2e):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_pair_potential(tps.GAUSS, v0, w.sigma)
        x0_dev.copy_(x0_host, non_blocking=True)
        lam, st = ctx.solve(w.k, tps.X_EVEN, 1e-12, w.block, evecs, x0=x0_dev, opts=opts,
                            stream=stream)
        evecs_host.copy_(evecs, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t += time.perf_counter() - t0
        e2e_pairs += passing_pairs(lam, ref)[0]
    E_T, E_pairs = aggregate(e2e_t, e2e_pairs, world, device="cuda")

    # solver variants on the same input: FP64-only and mixed, FP64 H-applies on the
    # tensor cores (default) or on the FP64 FMA pipe
    def variant_rate(h_dtype, h64_dtype, reps, graph=0):
        o = tps.default_opts()
        o.h_dtype = h_dtype
        o.h64_dtype = h64_dtype
        o.graph = graph
        step(o)
        ts, ok = [], True
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev0.record(stream)
            lam_v, _ = step(o)
            ev1.record(stream)
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1) / 1000.0)
            ok = ok and passing_pairs(lam_v, ref)[0] == len(ref)
        return passing_pairs(lam_v, ref)[0] / (sum(ts) / len(ts)), ok
    reps = max(1, min(3, args.steps))
    variants = {"fp64_tc (default, per-kernel timers on)": value / world}
    for name, hd, h64 in (("fp64_tc", tps.F64, tps.F64_TC), ("fp64_fma", tps.F64, tps.F64),
                          ("mixed_fp32_then_fp64_tc", tps.F32, tps.F64_TC),
                          ("mixed_fp32_then_fp64_fma", tps.F32, tps.F64)):
        variants[name], ok = variant_rate(hd, h64, reps)
        variants[name + "_all_pass"] = ok
    variants["fp64_tc_graph"], ok = variant_rate(tps.F64, tps.F64_TC, reps, graph=1)
    variants["fp64_tc_graph_all_pass"] = ok
    h2d = 8 * N + 8 * w.block * N
    d2h = 8 * w.k * N + 8 * w.k

    # batched sweep: the 256 independent instances of uneven grid size solved concurrently
    sweep = sweep_graph = None
    if rank == 0 and not args.no_sweep:
        sweep = run_sweep(tps, torch, args.sweep_streams)
        sweep_graph = run_sweep(tps, torch, args.sweep_streams, graph=1)
    apply_2d = run_apply_2d(tps, torch) if rank == 0 and not args.no_sweep else None

    # per-kernel rates from the solver's own CUDA-event timers over the timed solves; the
    # kernel family with the largest share of the step is the roofline
    pk = measured_peaks()
    fp64_peak = N_SM * FP64_FLOP_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    fp32_peak = N_SM * 256 * SM_MAX_MHZ * 1e6 / 1e12
    bf16_peak = pk.get("bf16_tflops_sustained")
    hbm_peak = pk.get("hbm_gbs")
    tot = lambda f: sum(getattr(st, f) for st in stats)
    step_s = local_t
    nx_s, ny = w.n[0] // 2 + 1, w.n[1]
    fp64_per_vec = 2.0 * nx_s * ny * (nx_s + ny) + 3.0 * nx_s * ny
    tc_per_vec = 2.0 * TC_PAIRS * nx_s * ny * (nx_s + ny)
    kernels = {}
    h_ms, h_fl = tot("h_ms"), tot("h_flops")
    if h_ms > 0:
        tflops = h_fl / fp64_per_vec * tc_per_vec / (h_ms / 1000.0) / 1e12
        kernels["k_oz_gemm"] = {
            "what": "FP64 H-apply on tcgen05 (BF16 digit products, exact FP32 levels; with its "
                    "digit-splitting kernels)",
            "bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": tflops / bf16_peak if bf16_peak else None,
            "peak_note": "bf16_tflops_sustained of measured (cuBLAS bf16, seconds-long loop)",
            "fp64_equivalent_tflops": h_fl / (h_ms / 1000.0) / 1e12,
            "vectors_per_launch": tot("h_applies") / max(tot("h_launches"), 1),
            "launches": tot("h_launches"), "share": h_ms / 1000.0 / step_s}
    # every 4th Gram / update / Ritz launch is timed (stats doc): rates come from the timed
    # launches, the share of the step is scaled up to all launches
    ms, fl, by = tot("gram_ms"), tot("gram_flops"), tot("gram_bytes")
    n_all = tot("gram_launches")
    n_timed = sum((st_.gram_launches + 3) // 4 for st_ in stats)
    if ms > 0:
        a = fl / (ms / 1000.0) / 1e12
        gbs = by / (ms / 1000.0) / 1e9
        kernels["k_gram"] = {
            "what": "FP64-accurate Gram products G = A^T B: digit-split BF16 products "
                    "(k_gram_split, mma.sync, exponents per 64-row block) for blocks of >= 1e5 "
                    "rows, FP64 FMA (k_gram) below; algorithmic bytes 8 nrows (p + q)",
            "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": gbs / hbm_peak if hbm_peak else None,
            "peak_note": "hbm_gbs of measured (STREAM-style copy)",
            "fp64_equivalent_tflops": a,
            "fp64_pipe_frac": a / fp64_peak,
            "fp64_pipe_note": "FP64-equivalent rate against the FP64 FMA pipe "
                              "(4 flop/clk/SM x 152 SMs x 2070 MHz, nominal-derived)",
            "launches": n_all, "timed_launches": n_timed,
            "share": ms * n_all / max(n_timed, 1) / 1000.0 / step_s}
    ms, fl, by = tot("upd_ms"), tot("upd_flops"), tot("upd_bytes")
    n_all = tot("upd_launches")
    n_timed = sum((st_.upd_launches + 3) // 4 for st_ in stats)
    if ms > 0:
        gbs = by / (ms / 1000.0) / 1e9
        kernels["k_update"] = {
            "what": "FP64-accurate block updates C = bC + a A Y: digit-split BF16 products "
                    "(k_update_split, mma.sync) for blocks of >= 1e5 rows, FP64 FMA (k_update) "
                    "below; algorithmic bytes 8 nrows (p + q), + 8 nrows q when C is read",
            "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": gbs / hbm_peak if hbm_peak else None,
            "peak_note": "hbm_gbs of measured (STREAM-style copy)",
            "fp64_equivalent_tflops": fl / (ms / 1000.0) / 1e12,
            "bf16_digit_tflops": SPLIT_UPDATE_PAIRS * fl / (ms / 1000.0) / 1e12,
            "bf16_digit_note": f"{SPLIT_UPDATE_PAIRS} BF16 digit-pair products per FP64 "
                               "multiply-add on mma.sync, counted as if every launch were split",
            "launches": n_all, "timed_launches": n_timed,
            "share": ms * n_all / max(n_timed, 1) / 1000.0 / step_s}
    rr_ms, rr_n, rr_t = tot("rr_ms"), tot("rr_launches"), tot("rr_timed")
    if rr_ms > 0 and rr_t > 0:
        kernels["k_rr_mixed"] = {
            "what": "Rayleigh-Ritz eigensolver of the projected m x m matrix (one 8-CTA "
                    "cluster; latency-bound, no throughput roofline)",
            "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
            "us_per_call": 1000.0 * rr_ms / rr_t, "launches": rr_n, "timed_launches": rr_t,
            "share": rr_ms * rr_n / rr_t / 1000.0 / step_s}
    p_ms, h32_ms = tot("prec_ms"), tot("h32_ms")
    if p_ms > 0:
        # the solver's default preconditioner: four TF32 mode products on tcgen05 (with the
        # FP64 -> FP32 conversion of its input); TF32 peak = measured BF16 x nominal 1.1/2.25
        a = tot("prec_flops") / (p_ms / 1000.0) / 1e12
        tf32_peak = bf16_peak * TF32_PER_BF16 if bf16_peak else None
        kernels["k_tf32_gemm"] = {"what": "preconditioner mode products, TF32 on tcgen05",
                                  "bound": "tensor", "achieved": a, "peak": tf32_peak,
                                  "unit": "TFLOP/s", "frac": a / tf32_peak if tf32_peak else None,
                                  "peak_note": "bf16_tflops_sustained of measured x 1.1/2.25 "
                                               "(nominal TF32 / BF16 dense ratio)",
                                  "launches": tot("prec_launches"),
                                  "share": p_ms / 1000.0 / step_s}
    if h32_ms > 0:
        a = tot("h32_flops") / (h32_ms / 1000.0) / 1e12
        kernels["k_gemm<float>"] = {"what": "FP32 mode products (FP32 H-apply of the mixed solver)",
                                    "bound": "alu", "achieved": a, "peak": fp32_peak,
                                    "unit": "TFLOP/s", "frac": a / fp32_peak,
                                    "peak_note": "FP32 FMA pipe, nominal-derived",
                                    "launches": tot("h32_launches"),
                                    "share": h32_ms / 1000.0 / step_s}
    with_roof = [k for k in kernels if kernels[k].get("frac") is not None]
    dom = max(with_roof, key=lambda k: kernels[k]["share"]) if with_roof else None
    roofline = None
    if dom is not None:
        kd = kernels[dom]
        launches = kd["launches"]
        roofline = {"bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                    "unit": kd["unit"], "frac": kd["frac"],
                    "traffic": traffic_per_launch(dom, kd), "kernel": dom,
                    "peak_note": kd["peak_note"], "launches": launches,
                    "time_share_of_step": kd["share"]}
    clocks = clk.summary()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores = cpu_oracle_sample(w, gold["v0"])
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle LOBPCG (NumPy/SciPy FP64) for the lowest x-even eigenpair of "
                         f"the same n=512 workload, {dt:.1f} s on the host; the 8-pair solve is "
                         f"not run (LOBPCG's cost grows at least linearly with the block, so "
                         f"8 pairs would take >= {8 * dt:.0f} s: this per-pair rate is an upper "
                         f"bound of the oracle's 8-pair rate)",
               "blas_threads": blas_threads()}
        cpu.update(cpu_oracle_legs(w, gold["v0"]))
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1000.0 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, world),
            "implementation": "FP64-accurate results: H mode products and tall block updates as "
                              "digit-split BF16 tensor-core products (tcgen05 / mma.sync), TF32 "
                              "tensor-core preconditioner, FP64 Gram/Ritz/orthogonalisation",
            "solver_variants": dict(variants, note="eigenpairs/s per GPU; tc = FP64 H-applies "
                                                   "on the tensor cores, fma = on the FP64 pipe; "
                                                   "graph = the outer loop as one captured CUDA "
                                                   "graph (tps_solver_opts.graph)"),
            "roofline": roofline,
            "kernels": kernels,
            "e2e": {"value": E_pairs / E_T, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": n_e2e},
            "clocks": clocks,
            "gpu_launches": int(sum(st.kernel_launches for st in stats)),
            "eigen_rel_err_max": rel_max, "pairs_passing": total_pairs,
            "solve_time_stats": solve_stats, "setup": setup,
            "solver": {"outer_iters": stats[-1].outer_iters, "h_applies": stats[-1].h_applies,
                       "prec_applies": stats[-1].prec_applies, "restarts": stats[-1].restarts},
            "wall_s": wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if sweep is not None:
            line["sweep"] = sweep
        if sweep_graph is not None:
            line["sweep_graph"] = sweep_graph
        if apply_2d is not None:
            line["h_apply_2d"] = apply_2d
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
