"""Learned warm start: data generation from the solver's own eigenvectors, training on the
GPU (tps_ws_loss_grad / tps_ws_adam_step), and its evaluation against a cold start and the
non-learned homotopy start (the previous point of a decreasing-E0 sweep).

Every numerical step runs in the library's kernels; this module only sequences them.  The
one exception is training-data preparation in 2D: the square grid keeps pairs of states
exactly degenerate, and the 2 x 2 rotation that makes their targets well defined is taken
on the host on the px x py coefficient matrices (canonical_targets).
"""
from __future__ import annotations

import time

import numpy as np

from . import tps


def parity_of(inst):
    """The sector solved: the x-even states in 1D, every state in 2D."""
    return tps.X_EVEN if inst.get("dim", 1) == 1 else tps.ANY


def pair_v0(inst, E0=None):
    """Well depth binding the heavy-light pair by E0 (default the instance's)."""
    mu = inst["M"] * inst["m"] / (inst["M"] + inst["m"])
    return tps.two_body_v0(inst.get("dim", 1), mu, 1.0, inst["E0"] if E0 is None else E0,
                           tps.GAUSS, inst["sigma"], inst["n"], inst["L"])


def make_context(inst, device=0):
    """Context for one instance (dict with M, m, E0, sigma, n, L and optionally dim, default
    1; n points and half-width L on every Cartesian component); returns (ctx, v0)."""
    dim = inst.get("dim", 1)
    ctx = tps.Context(dim, device)
    ctx.set_masses(inst["M"], inst["m"], 1.0)
    ctx.set_grid([inst["n"]] * 2 * dim, [inst["L"]] * 2 * dim)
    v0 = pair_v0(inst)
    ctx.set_pair_potential(tps.GAUSS, v0, inst["sigma"])
    return ctx, v0


def _reflection_signs(q):
    # real Fourier modes 1, cos, sin, cos 2, sin 2, ...: F_a(-x) = +F_a(x) unless a is a sine
    return np.array([-1.0 if a > 0 and a % 2 == 0 else 1.0 for a in range(q)])


def canonical_targets(T, lam, px, py, rel=1e-9):
    """2D training targets with exactly degenerate eigenvalues made well defined: the
    solver returns an arbitrary orthonormal basis of such an eigenspace, so each cluster's
    targets are rotated onto eigenvectors of the reflection (x1, y1) -> (-x1, -y1) (a
    symmetry of H and of the grid), the even one first.  T: [k, px, py] torch; returns a
    new torch tensor on the same device."""
    import scipy.linalg
    import torch
    qx, qy = int(round(px ** 0.5)), int(round(py ** 0.5))
    sign = np.outer(np.repeat(_reflection_signs(qx), qx), np.repeat(_reflection_signs(qy), qy))
    Tn = T.detach().cpu().numpy().astype(np.float64)
    k, i = len(lam), 0
    while i < k:
        j = i + 1
        while j < k and abs(lam[j] - lam[i]) <= rel * max(abs(lam[i]), abs(lam[0])):
            j += 1
        if j - i > 1:
            G = Tn[i:j].reshape(j - i, -1)
            R = (G * sign.ravel()) @ G.T
            w, V = scipy.linalg.eigh(0.5 * (R + R.T), G @ G.T)
            Tn[i:j] = (V[:, np.argsort(-w)].T @ G).reshape(j - i, px, py)
        i = j
    return torch.from_numpy(Tn.astype(np.float32)).to(T.device)


def make_dataset(model, instances, k, block=None, nstreams=8, device=0, chunk=256):
    """Solve every instance (k lowest x-even pairs, cold start, batched `chunk` instances at
    a time) and project the eigenvectors onto the model's basis.  Returns (X [n*k, 4]
    float32 torch, T [n*k, px, py] float32 torch, total solve seconds)."""
    import torch
    block = block or k
    Xs, Ts, dt = [], [], 0.0
    for c0 in range(0, len(instances), chunk):
        part = instances[c0: c0 + chunk]
        ctxs, v0s = zip(*[make_context(i, device) for i in part])
        evecs = [torch.empty(k, c.info()[0], dtype=torch.float64, device="cuda") for c in ctxs]
        t0 = time.perf_counter()
        lam, stats, status = tps.solve_batch(list(ctxs), [k] * len(ctxs), parity_of(part[0]),
                                             1e-12, block, evecs, nstreams=nstreams)
        torch.cuda.synchronize()
        dt += time.perf_counter() - t0
        if any(s != tps.OK for s in status):
            raise RuntimeError("a training solve failed")
        Xs.append(np.concatenate([model.features([i["M"] / i["m"]] * k, [v] * k,
                                                 [i["sigma"]] * k, list(range(k)))
                                  for i, v in zip(part, v0s)]))
        T = [model.project(c, e) for c, e in zip(ctxs, evecs)]
        if part[0].get("dim", 1) == 2:
            T = [canonical_targets(t, l, model.px, model.py) for t, l in zip(T, lam)]
        Ts.append(torch.cat(T))
        torch.cuda.synchronize()
        for c in ctxs:
            c.close()
        del evecs
    return torch.from_numpy(np.concatenate(Xs)).cuda(), torch.cat(Ts), dt


def train(model, X, T, steps=2000, batch=256, lr=1e-3, lr_final=1e-4, seed=0):
    """Adam on random mini-batches with a geometric learning-rate decay; returns the loss
    history (one value per step)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    losses = []
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).cuda()
        xb, tb = X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous()
        loss, _ = model.loss_grad(xb, tb)
        rate = lr * (lr_final / lr) ** (s / max(1, steps - 1))
        model.adam_step(lr=rate)
        losses.append(loss)
    return losses


HOMOTOPY_STEP = 1.25  # E0 ratio between neighbouring points of a decreasing-E0 sweep


def homotopy_solve(ctx, inst, k, block, tol, ev, step=HOMOTOPY_STEP, timed=True):
    """The non-learned baseline (Sec. 6, homotopy over E0): solve the neighbouring point of
    a sweep that decreases E0 -- the same M/m, sigma and grid, E0 larger by `step`, v0 tuned
    to it -- and start the instance's solve from its k eigenvectors.  The neighbour's solve
    is the previous step of the sweep and is not timed.  Returns (eigenvalues, Stats,
    seconds of the instance's solve); the context's potential is the instance's after."""
    import torch
    v_prev, v_inst = pair_v0(inst, inst["E0"] * step), pair_v0(inst)
    prev = torch.empty_like(ev)
    ctx.set_pair_potential(tps.GAUSS, v_prev, inst["sigma"])
    ctx.solve(k, parity_of(inst), tol, block, prev)
    ctx.set_pair_potential(tps.GAUSS, v_inst, inst["sigma"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, st = ctx.solve(k, parity_of(inst), tol, block, ev, x0=prev)
    torch.cuda.synchronize()
    return lam, st, time.perf_counter() - t0


def evaluate(model, instances, k, block=None, tol=1e-12, device=0, homotopy=True):
    """Cold start, learned warm start and (homotopy=True) the homotopy start on each
    instance: outer iterations, H applications (MVMs, the paper's Table 2 count), solve
    time and the largest relative eigenvalue difference to the cold solve (the tests check
    the eigenpairs with the oracle)."""
    import torch
    block = block or k
    rows = []
    for inst in instances:
        ctx, v0 = make_context(inst, device)
        ev = torch.empty(k, ctx.info()[0], dtype=torch.float64, device="cuda")
        out = {}
        for name, m in (("cold", None), ("warm", model)):
            tps.solve_warm(m, ctx, inst["M"] / inst["m"], v0, inst["sigma"], k, parity_of(inst),
                           tol, block, ev)  # warm-up (builds the sector operator and workspaces)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lam, st, used = tps.solve_warm(m, ctx, inst["M"] / inst["m"], v0, inst["sigma"], k,
                                           parity_of(inst), tol, block, ev)
            torch.cuda.synchronize()
            out[name] = (lam, st.outer_iters, time.perf_counter() - t0, used, st.h_applies)
        lc, lw = out["cold"][0], out["warm"][0]
        scale = np.maximum(np.abs(lc), abs(lc[0]))
        row = {"cold_iters": out["cold"][1], "warm_iters": out["warm"][1],
               "cold_s": out["cold"][2], "warm_s": out["warm"][2],
               "cold_mvm": out["cold"][4], "warm_mvm": out["warm"][4],
               "used_warm": out["warm"][3],
               "rel_diff": float(np.max(np.abs(lc - lw) / scale))}
        if homotopy:
            lh, sth, th = homotopy_solve(ctx, inst, k, block, tol, ev)
            row.update({"homotopy_iters": sth.outer_iters, "homotopy_mvm": sth.h_applies,
                        "homotopy_s": th,
                        "homotopy_rel_diff": float(np.max(np.abs(lc - lh) / scale))})
        ctx.close()
        rows.append(row)
    return rows


TWO_D = dict(ratio=(5.0, 30.0), E0=(0.1, 1.0), sigmas=(1.0,), L=10.0, dim=2)


def _arm(model, train_set, test_set, k, eval_k, steps, chunk):
    """Train `model` on the eigenvectors of train_set, evaluate on test_set (dict of the
    training and evaluation figures)."""
    import torch
    t0 = time.perf_counter()
    X, T, solve_s = make_dataset(model, train_set, k=k, nstreams=16, chunk=chunk)
    t1 = time.perf_counter()
    losses = train(model, X, T, steps=steps, batch=256, lr=2e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rows = evaluate(model, test_set, k=eval_k)
    mean = lambda key: float(np.mean([r[key] for r in rows]))
    return {
        "train": {"instances": len(train_set), "n": sorted({i["n"] for i in train_set}),
                  "eigenvectors": int(X.shape[0]), "data_s": t1 - t0, "solve_s": solve_s,
                  "train_s": t2 - t1, "steps": steps, "loss_first": float(np.mean(losses[:20])),
                  "loss_last": float(np.mean(losses[-20:]))},
        "eval": {"instances": len(rows), "n": test_set[0]["n"], "k": eval_k,
                 "cold_iters": mean("cold_iters"), "warm_iters": mean("warm_iters"),
                 "homotopy_iters": mean("homotopy_iters"),
                 "cold_mvm": mean("cold_mvm"), "warm_mvm": mean("warm_mvm"),
                 "homotopy_mvm": mean("homotopy_mvm"),
                 "cold_ms": 1e3 * mean("cold_s"), "warm_ms": 1e3 * mean("warm_s"),
                 "homotopy_ms": 1e3 * mean("homotopy_s"),
                 "homotopy_step": HOMOTOPY_STEP,
                 "used_warm": sum(r["used_warm"] for r in rows),
                 "max_rel_diff": max(r["rel_diff"] for r in rows),
                 "homotopy_max_rel_diff": max(r["homotopy_rel_diff"] for r in rows)}}


def main(argv=None):
    """Train models on solver eigenvectors (1D: the sweep generator; 2D: instances on a
    coarser grid than the evaluation's) and compare learned, homotopy and cold starts on
    unseen instances; prints one JSON line."""
    import argparse
    import json
    from .inputs import warmstart_instances
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train-instances", type=int, default=2500)
    ap.add_argument("--k", type=int, default=8, help="eigenvectors per training instance")
    ap.add_argument("--eval-instances", type=int, default=512)
    ap.add_argument("--eval-n", type=int, default=256)
    ap.add_argument("--eval-k", type=int, default=4)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--px", type=int, default=32)
    ap.add_argument("--py", type=int, default=32)
    ap.add_argument("--train-2d-instances", type=int, default=400,
                    help="2D training instances (0: no 2D arm)")
    ap.add_argument("--train-2d-n", type=int, default=24)
    ap.add_argument("--k-2d", type=int, default=6)
    ap.add_argument("--eval-2d-instances", type=int, default=32)
    ap.add_argument("--eval-2d-n", type=int, default=40)
    ap.add_argument("--q-2d", type=int, default=7,
                    help="Fourier modes per Cartesian component in 2D (px = py = q^2)")
    args = ap.parse_args(argv)
    out = {}
    if args.train_instances > 0:
        model = tps.WarmStart(px=args.px, py=args.py, rank=16, hidden=256, seed=1)
        out["1d"] = _arm(model, warmstart_instances(args.train_instances, seed=21),
                         warmstart_instances(args.eval_instances, seed=22, ns=(args.eval_n,)),
                         args.k, args.eval_k, args.steps, 256)
        model.close()
    if args.train_2d_instances > 0:
        q2 = args.q_2d * args.q_2d
        model = tps.WarmStart(px=q2, py=q2, rank=16, hidden=256, seed=1)
        out["2d"] = _arm(model, warmstart_instances(args.train_2d_instances, seed=23,
                                                    ns=(args.train_2d_n,), **TWO_D),
                         warmstart_instances(args.eval_2d_instances, seed=24,
                                             ns=(args.eval_2d_n,), **TWO_D),
                         args.k_2d, args.eval_k, args.steps, 64)
        model.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
