"""Write oracle eigenvalues for the full-size workloads into tests/golden/*.json.

Calls only oracle/ (never the CUDA path).  Usage: python tests/golden/make_golden.py [name ...]
  1d_n512 : M/m = 40, n = 512 per coordinate on [-20, 20), v0 tuned to E0 = 1e-3 on the
            y grid (heavy-light reduced mass), sigma = 1, 8 lowest x-even eigenpairs.
  2d_n16  : 2D, M/m = 20, n = 16 per component on [-10, 10), v0 = 2, 4 lowest pairs.
  2d_n24  : 2D, M/m = 20, n = 24 per component on [-12, 12), v0 = 2, 4 lowest pairs.
  sweep   : the 256 instances of inputs.sweep_instances(), 4 lowest x-even pairs each.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.hamiltonian import problem_1d, problem_2d, GAUSS, coefficients_from_masses  # noqa: E402
from oracle.two_body import tune_v0  # noqa: E402
from oracle.eig import lowest_iterative, residual_norms  # noqa: E402
from oracle.sector import X_EVEN, ANY  # noqa: E402
from paper_2111_02534_gb300.inputs import WORKLOADS  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def make_1d_n512():
    w = WORKLOADS["1d_n512"]
    _, _, mu_hl = coefficients_from_masses(w.M, w.m, w.hbar)
    v0 = tune_v0(w.E0, mu_hl, w.sigma, GAUSS, w.n[1], w.L[1], hbar=w.hbar)
    P = problem_1d(w.M, w.m, w.hbar, w.n, w.L, v0, w.sigma)
    t = time.time()
    lam, X = lowest_iterative(P, w.k, X_EVEN, tol=1e-13, extra=6)
    res = residual_norms(P, X, lam) / P.norm_estimate()
    return {"workload": w.name, "v0": v0, "evals": lam.tolist(), "rel_resid": res.tolist(),
            "hnorm_est": P.norm_estimate(), "seconds": time.time() - t,
            "method": "oracle.eig.lowest_iterative (LOBPCG), x-even sector"}


def make_2d_n16():
    # 2D at a grid the oracle can finish: 16 points per component on [-10, 10)
    P = problem_2d(20.0, 1.0, 1.0, (16, 16, 16, 16), (10.0,) * 4, 2.0, 1.0)
    t = time.time()
    lam, X = lowest_iterative(P, 4, ANY, tol=1e-12, extra=6)
    res = residual_norms(P, X, lam) / P.norm_estimate()
    return {"workload": "2d_n16", "M": 20.0, "m": 1.0, "n": [16] * 4, "L": [10.0] * 4,
            "v0": 2.0, "sigma": 1.0, "evals": lam.tolist(), "rel_resid": res.tolist(),
            "seconds": time.time() - t, "method": "oracle.eig.lowest_iterative (LOBPCG), all states"}


def make_2d_n24():
    # 2D between the oracle-checked 16^4 and the 48^4 workload: 24 points per component
    # on [-12, 12) (331,776 unknowns)
    P = problem_2d(20.0, 1.0, 1.0, (24, 24, 24, 24), (12.0,) * 4, 2.0, 1.0)
    t = time.time()
    lam, X = lowest_iterative(P, 4, ANY, tol=1e-12, extra=6)
    res = residual_norms(P, X, lam) / P.norm_estimate()
    return {"workload": "2d_n24", "M": 20.0, "m": 1.0, "n": [24] * 4, "L": [12.0] * 4,
            "v0": 2.0, "sigma": 1.0, "evals": lam.tolist(), "rel_resid": res.tolist(),
            "seconds": time.time() - t, "method": "oracle.eig.lowest_iterative (LOBPCG), all states"}


def _sweep_one(args):
    import os
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    i, inst = args
    _, _, mu_hl = coefficients_from_masses(inst["M"], inst["m"], 1.0)
    v0 = tune_v0(inst["E0"], mu_hl, inst["sigma"], GAUSS, inst["n"], inst["L"])
    P = problem_1d(inst["M"], inst["m"], 1.0, (inst["n"], inst["n"]), (inst["L"], inst["L"]), v0,
                   inst["sigma"])
    lam, X = lowest_iterative(P, 4, X_EVEN, tol=1e-13, extra=4, seed=i)
    res = residual_norms(P, X, lam) / P.norm_estimate()
    return {"index": i, **inst, "v0": v0, "evals": lam.tolist(), "rel_resid": res.tolist()}


def make_sweep():
    # the 256-instance sweep: 4 lowest x-even eigenpairs per instance
    import multiprocessing as mp
    from paper_2111_02534_gb300.inputs import sweep_instances
    insts = sweep_instances()
    t = time.time()
    with mp.get_context("spawn").Pool(int(os.environ.get("GOLDEN_PROCS", "8"))) as pool:
        out = pool.map(_sweep_one, list(enumerate(insts)), chunksize=1)
    return {"workload": "sweep", "count": len(out), "instances": out, "evals": [o["evals"] for o in out],
            "seconds": time.time() - t,
            "method": "oracle.eig.lowest_iterative (LOBPCG), x-even sector, 4 pairs per instance"}


MAKERS = {"1d_n512": make_1d_n512, "2d_n16": make_2d_n16, "2d_n24": make_2d_n24,
          "sweep": make_sweep}

if __name__ == "__main__":
    names = sys.argv[1:] or list(MAKERS)
    for name in names:
        out = MAKERS[name]()
        with open(os.path.join(HERE, f"evals_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, out["evals"], "%.0fs" % out["seconds"])
