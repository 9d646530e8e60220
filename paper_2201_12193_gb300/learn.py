"""Learned troubled-cell indicator: label harvest, training, judge.

All arithmetic runs in the library's CUDA kernels (features, BF16 tensor-core
forward/backward, Adam); this module only schedules them.  Labels are the
paper's KXRCF decisions (eq. (KXRCF_)) on the first-stage input of steps of the
method itself; KXRCF stays the fallback for low-confidence cells and the judge.

  python -m paper_2201_12193_gb300.learn train      # writes data/mlp_indicator.npz
  python -m paper_2201_12193_gb300.learn judge
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import hweno, workloads as W


def init_params(seed=0):
    """He-normal weights, zero biases, in the flat layout of include/hweno.h."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2 / 108), 64 * 108), np.zeros(64), rng.normal(0, math.sqrt(2 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, math.sqrt(1 / 64), 64), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "mlp_indicator.npz")


def training_problems(seed=0, n=256, count=6, ncircles=4):
    """Blast-circle and four-quadrant problems (the workload's data families)."""
    probs = []
    for k in range(count):
        if k % 2 == 0:
            probs.append(W.blast_2d(n, seed=seed * 1000 + k, ncircles=ncircles))
        else:
            probs.append(W.four_quadrant_2d(n, seed=seed * 1000 + k))
    return probs


# Default training recipe: blast data of the C4 family (8 circles) at three
# resolutions plus four-quadrant Riemann data, so that the network sees the
# h^2 scale of its features vary.  (grid size, blast seeds, four-quadrant seeds, steps)
RECIPE = ((256, 6, 2, 40), (512, 4, 2, 30), (1024, 2, 0, 24))


def recipe_problems(seed=1):
    out = []
    for n, nb, nq, steps in RECIPE:
        for k in range(nb):
            out.append((W.blast_2d(n, seed=seed * 10000 + n + k, ncircles=8), steps))
        for k in range(nq):
            out.append((W.four_quadrant_2d(n, seed=seed * 10000 + n + 100 + k), steps))
    return out


def harvest(problems, steps=12, neg_ratio=3, seed=0, pos_weight=1.0, max_pos=20000):
    """(X, y, w) on the GPU: the KXRCF-flagged cells of the first stage of each
    step (at most max_pos per step, drawn at random), plus unflagged cells (half
    next to flagged ones, half anywhere); class weights balance the two labels,
    the troubled class then scaled by pos_weight (missing a troubled cell costs
    more than a false alarm).  problems: Problem objects or (Problem, steps)."""
    import torch
    rng = np.random.default_rng(seed)
    Xs, ys = [], []
    for item in problems:
        p, nsteps = item if isinstance(item, tuple) else (item, steps)
        s = hweno.Solver.from_problem(p)
        s.set_positivity_check(False)     # the scheme's own transient p < 0 averages carry on
        s.set_moments(torch.from_numpy(p.m).cuda())
        U = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        for _ in range(nsteps):
            s.get_moments(U)
            Uc = U.clone()
            try:
                s.step(s.max_dt(0.6))
                mask = s.troubled_mask()[0].reshape(-1)
            except hweno.HwenoError:
                break
            pos = np.flatnonzero(mask)
            if len(pos) > max_pos:
                pos = rng.choice(pos, max_pos, replace=False)
            neg_all = np.flatnonzero(mask == 0)
            if len(neg_all) == 0:
                continue
            near = np.zeros_like(mask, dtype=bool)
            m2 = mask.reshape(p.ny, p.nx).astype(bool)
            for sh in ((0, 1), (0, -1), (1, 1), (1, -1)):
                near |= np.roll(m2, sh[1], axis=sh[0]).reshape(-1)
            hard = np.flatnonzero(near & (mask == 0))
            k = max(len(pos), 64)
            neg = np.concatenate([rng.choice(hard, min(len(hard), k * neg_ratio // 2), replace=False)
                                  if len(hard) else np.zeros(0, np.int64),
                                  rng.choice(neg_all, min(len(neg_all), k * neg_ratio // 2), replace=False)])
            cells = np.concatenate([pos, neg]).astype(np.int32)
            X = torch.empty((len(cells), 108), dtype=torch.float32, device="cuda")
            s.features(Uc, torch.from_numpy(cells).cuda(), X)
            Xs.append(X)
            ys.append(torch.from_numpy(np.concatenate([np.ones(len(pos)), np.zeros(len(neg))]).astype(np.float32)).cuda())
        s.close()
    X = torch.cat(Xs)
    y = torch.cat(ys)
    npos = float(y.sum())
    nneg = float(len(y) - npos)
    w = torch.where(y > 0.5, pos_weight * 0.5 * len(y) / max(npos, 1.0), 0.5 * len(y) / max(nneg, 1.0)).float()
    return X, y, w


def train(X, y, w, epochs=20, batch=8192, lr=2e-3, seed=0, params=None, log=None):
    """Adam on the weighted mean BCE with the library's tensor-core kernels;
    the step size follows a cosine from lr down to lr/20."""
    import torch
    th = torch.from_numpy(init_params(seed) if params is None else params).cuda()
    m1 = torch.zeros_like(th)
    m2 = torch.zeros_like(th)
    grad = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(seed)
    n = X.shape[0]
    step = 0
    hist = []
    total = epochs * ((n + batch - 1) // batch)
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            Xb, yb, wb = X[idx].contiguous(), y[idx].contiguous(), w[idx].contiguous()
            grad.zero_()
            loss.zero_()
            hweno.mlp_loss_grad(th, Xb, yb, wb, grad, loss)
            step += 1
            hweno.mlp_adam(th, grad, m1, m2, step, lr * (0.05 + 0.475 * (1 + math.cos(math.pi * step / total))))
            tot += float(loss.item()) * len(idx)
        hist.append(tot / n)
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return th.cpu().numpy(), hist


def predict(params, X):
    import torch
    th = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
    prob = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    hweno.mlp_forward(th, X, prob)
    return prob


def judge(params, problems, steps=10, conf=0.9):
    """Learned indicator against KXRCF on identical stage inputs along the learned
    run: recall, false-negative rate, false-positive rate, fraction of cells the
    network decided alone, and the relative L1 drift of the final state from the
    plain scheme's."""
    import torch
    tp = fp = fn = tn = 0
    cells_total = fallbacks = 0
    rer_ml = rer_kx = 0
    drift_num = drift_den = 0.0
    for p in problems:
        ml = hweno.Solver.from_problem(p, indicator="mlp")
        ml.set_mlp(params, conf)
        kx = hweno.Solver.from_problem(p)
        ml.set_positivity_check(False)
        kx.set_positivity_check(False)
        m0 = torch.from_numpy(p.m).cuda()
        ml.set_moments(m0)
        kx.set_moments(m0)
        U = torch.empty(ml.shape, dtype=torch.float64, device="cuda")
        Um = torch.empty_like(U)
        L = torch.empty_like(U)
        mk = torch.empty((p.ny, p.nx), dtype=torch.uint8, device="cuda")
        mm = torch.empty_like(mk)
        ok = True
        for _ in range(steps):
            ml.get_moments(U)
            ml.rhs(U, Um, L, mm)
            kx.rhs(U, Um, L, mk)
            torch.cuda.synchronize()
            a = mm.cpu().numpy().astype(bool)
            b = mk.cpu().numpy().astype(bool)
            tp += int((a & b).sum()); fp += int((a & ~b).sum()); fn += int((~a & b).sum()); tn += int((~a & ~b).sum())
            try:
                ml.step(kx.max_dt(0.6))
                kx.step(kx.max_dt(0.6))
            except hweno.HwenoError:
                ok = False
                break
        cells_total += p.nx * p.ny * 4 * steps        # rhs calls + 3 stages per step
        fallbacks += ml.mlp_fallbacks()
        rer_ml += ml.rerecon_count()
        rer_kx += kx.rerecon_count()
        if ok:
            a = ml.get_moments()
            b = kx.get_moments()
            drift_num += float(np.abs(a - b).sum())
            drift_den += float(np.abs(b).sum())
        ml.close()
        kx.close()
    return {"recall": tp / max(tp + fn, 1), "false_negative_rate": fn / max(tp + fn, 1),
            "false_positive_rate": fp / max(fp + tn, 1), "flagged_kxrcf": tp + fn, "flagged_mlp": tp + fp,
            "decided_by_network": 1.0 - fallbacks / max(cells_total, 1),
            "rerecon_cells_mlp": rer_ml, "rerecon_cells_kxrcf": rer_kx,
            "l1_drift_vs_kxrcf": drift_num / max(drift_den, 1e-300)}


def load_params(path=None):
    """The trained parameters (float32, flat layout of include/hweno.h)."""
    with np.load(path or PARAMS_FILE) as z:
        return np.ascontiguousarray(z["params"], dtype=np.float32)


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train", help="harvest KXRCF labels, train on the GPU, judge on held-out data")
    t.add_argument("--out", default=PARAMS_FILE)
    t.add_argument("--epochs", type=int, default=40)
    t.add_argument("--pos-weight", type=float, default=3.0)
    t.add_argument("--seed", type=int, default=1)
    j = sub.add_parser("judge", help="judge saved parameters on held-out blast data")
    j.add_argument("--params", default=PARAMS_FILE)
    j.add_argument("--n", type=int, default=1024)
    j.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    held = [W.blast_2d(1024, seed=900 + k, ncircles=8) for k in range(2)]
    if args.cmd == "judge":
        held = [W.blast_2d(args.n, seed=900 + k, ncircles=8) for k in range(2)]
        print(judge(load_params(args.params), held, steps=args.steps))
        return
    t0 = time.time()
    probs = recipe_problems(args.seed)
    X, y, w = harvest(probs, pos_weight=args.pos_weight, seed=args.seed)
    t_h = time.time() - t0
    print(f"harvest: {X.shape[0]} samples ({int(y.sum())} flagged) in {t_h:.1f} s")
    t0 = time.time()
    params, hist = train(X, y, w, epochs=args.epochs, batch=8192, lr=3e-3, seed=args.seed)
    t_t = time.time() - t0
    print(f"train: {t_t:.1f} s, loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    rep = judge(params, held, steps=10)
    print(rep)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=params, loss=np.array(hist), samples=X.shape[0], harvest_s=t_h, train_s=t_t,
             recipe=np.array(RECIPE), **{"judge_" + k: v for k, v in rep.items()})


if __name__ == "__main__":
    main()
