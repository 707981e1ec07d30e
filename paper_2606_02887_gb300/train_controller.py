"""Training of the learned step controller on the GPU.

Problems: seeded planted problems drawn like the uneven-batch workload (n ~ U{64..2048},
r ~ U{4..32}, 1% relative noise).  Two label sets:

  greedy   record-mode solves (step_controller = 2), several random restarts per problem in
           one batched solve.  At every inner step the solver follows the plain BB trajectory
           and records the state's features and the best of 9 candidate multipliers by the
           accepted one-step decrease; about `per_traj` records per trajectory are kept.
  rollout  rollout-branch solves (step_controller = 4): 9 restarts per group share a start and
           follow the plain BB trajectory up to one inner step (the branch point, drawn per
           solve), where restart c of the group scales the step by 2^((c - 4) / 2).  All of
           them then run plain BB to the end of the next outer iteration (10 to 19 further
           inner steps), and the label of the branch point's features is the multiplier whose
           restart ends with the lowest objective (ties go to the plain step, multiplier 1).

Training: snmf_mlp_train (hand-written forward/backward and Adam kernels).

    python -m paper_2606_02887_gb300.train_controller --labels rollout --problems 400

writes controller_weights.json next to this file.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import snmf as S

WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "controller_weights.json")
TRAIN_SEED_BASE = 900000  # problem seeds of the training set (evaluation uses other seeds)


def init_weights(seed: int = 0) -> np.ndarray:
    g = np.random.default_rng(seed)
    w = np.zeros(S.SNMF_MLP_NPARAMS, dtype=np.float32)
    n1 = S.SNMF_MLP_IN * S.SNMF_MLP_HIDDEN
    w[:n1] = g.normal(0.0, 1.0 / math.sqrt(S.SNMF_MLP_IN), n1)
    w[n1 + S.SNMF_MLP_HIDDEN:n1 + 2 * S.SNMF_MLP_HIDDEN] = g.normal(0.0, 0.1 / math.sqrt(S.SNMF_MLP_HIDDEN),
                                                                   S.SNMF_MLP_HIDDEN)
    return w


def load_weights(path: str = WEIGHTS_PATH) -> np.ndarray:
    d = json.load(open(path))
    return np.asarray(d["weights"], dtype=np.float32)


def collect(problems: int, restarts: int, per_traj: int = 20, seed_base: int = TRAIN_SEED_BASE,
            max_iter: int = 200, log=print):
    """Record-mode solves; returns (features [m, 5], targets [m])."""
    import torch

    from workloads import planted_dense, uniform_init

    dev = torch.device("cuda:0")
    g = np.random.default_rng(seed_base)
    feats, targs = [], []
    t0 = time.time()
    for p in range(problems):
        n = int(g.integers(64, 2049))
        r = int(g.integers(4, 33))
        A, _ = planted_dense(n, r, seed=seed_base + 1 + p, rel_noise=0.01)
        upper = math.sqrt(A.mean() / r)
        W0 = np.concatenate([uniform_init(n, r, upper, seed_base + 100000 + p * 64 + j) for j in range(restarts)], 1)
        At = torch.tensor(A, dtype=torch.float32, device=dev)
        Wt = torch.tensor(W0, dtype=torch.float32, device=dev)
        Ht = Wt.clone()
        o = S.snmf_default_options(precision=S.SNMF_F32, batch=restarts, step_controller=2, max_iter=max_iter,
                                   tol=1e-4, nonmonotone_M=10)
        h = S.snmf_create(S.dense_matrix(At), r, o)
        try:
            S.snmf_solve(h, Wt, Ht)
            f, t = S.snmf_controller_data(h)
        finally:
            S.snmf_destroy(h)
        keep = min(len(t), per_traj * restarts)
        if keep:
            sel = g.choice(len(t), keep, replace=False)
            feats.append(f[sel])
            targs.append(t[sel])
        if log and (p + 1) % 100 == 0:
            log(f"collected {p + 1}/{problems} problems, {sum(len(x) for x in targs)} samples, "
                f"{time.time() - t0:.1f} s")
    return np.concatenate(feats), np.concatenate(targs)


def rollout_labels(fvals: np.ndarray, rel_tie: float = 1e-12) -> np.ndarray:
    """Targets (log2 multipliers) of rollout groups: fvals[g][c] is the objective at the end
    of the rollout of group g's candidate c (multiplier 2^((c - 4) / 2)).  The label is the
    candidate with the lowest objective; a candidate must beat the plain step (c = 4) by more
    than rel_tie * |f_4| to be chosen, so ties go to multiplier 1.  Groups with a non-finite
    objective get NaN (dropped by the caller)."""
    f = np.asarray(fvals, dtype=np.float64)
    out = np.full(f.shape[0], np.nan)
    for g in range(f.shape[0]):
        row = f[g]
        if not np.all(np.isfinite(row)):
            continue
        best = int(np.argmin(row))
        if row[4] - row[best] <= rel_tie * abs(row[4]):
            best = 4
        out[g] = 0.5 * (best - 4)
    return out


def collect_rollout(problems: int, branches: int = 2, groups: int = 8, t_max: int = 80,
                    seed_base: int = TRAIN_SEED_BASE, log=print):
    """Rollout-branch solves; returns (features [m, 5], objectives [m, 9], relative projected
    gradients [m, 9]) of the m recorded branch points, each row of the last two over the nine
    candidates at the end of the rollout."""
    import torch

    from workloads import planted_dense, uniform_init

    dev = torch.device("cuda:0")
    g = np.random.default_rng(seed_base + 7)
    K = 5  # inner steps per block (the library default)
    feats, fv, pv = [], [], []
    t0 = time.time()
    for p in range(problems):
        n = int(g.integers(64, 2049))
        r = int(g.integers(4, 33))
        A, _ = planted_dense(n, r, seed=seed_base + 1 + p, rel_noise=0.01)
        upper = math.sqrt(A.mean() / r)
        m = max(1, min(groups, 4096 // (9 * r)))
        b = 9 * m
        starts = [uniform_init(n, r, upper, seed_base + 100000 + p * 64 + q) for q in range(m)]
        W0 = np.concatenate([starts[q] for q in range(m) for _ in range(9)], 1)
        At = torch.tensor(A, dtype=torch.float32, device=dev)
        for _ in range(branches):
            t = int(g.integers(0, t_max))
            blk = int(g.integers(0, 2))
            k = int(g.integers(0, K - 1))  # the multiplier of the block's last step has no effect
            o = S.snmf_default_options(precision=S.SNMF_F32, batch=b, step_controller=4,
                                       branch_step=2 * t * K + blk * K + k, max_iter=t + 2, tol=0.0,
                                       nonmonotone_M=10, inner_iters=K)
            Wt = torch.tensor(W0, dtype=torch.float32, device=dev)
            Ht = Wt.clone()
            h = S.snmf_create(S.dense_matrix(At), r, o)
            try:
                S.snmf_solve(h, Wt, Ht)
                f, grp = S.snmf_controller_data(h, capacity=m)
                per = S.snmf_restart_stats(h, b)
            finally:
                S.snmf_destroy(h)
            fin, pg = per["f"].reshape(m, 9), per["pg_rel"].reshape(m, 9)
            for row, q in zip(f, grp.astype(int)):
                if 0 <= q < m and np.all(np.isfinite(row)):
                    feats.append(row)
                    fv.append(fin[q])
                    pv.append(pg[q])
        if log and (p + 1) % 50 == 0:
            log(f"rollouts: {p + 1}/{problems} problems, {len(fv)} samples, {time.time() - t0:.1f} s")
    return (np.asarray(feats, dtype=np.float32).reshape(-1, S.SNMF_MLP_IN), np.asarray(fv).reshape(-1, 9),
            np.asarray(pv).reshape(-1, 9))


def rollout_targets(feats, fvals, pgvals, score: str = "f", margin: float = 1e-12):
    """Training pairs from collect_rollout's output: labels by the end-of-rollout objective
    (score "f") or relative projected gradient (score "pg"), a candidate having to beat the
    plain step by more than `margin` relative; rows with a non-finite label are dropped."""
    lab = rollout_labels(fvals if score == "f" else pgvals, rel_tie=margin)
    ok = np.isfinite(lab)
    return np.asarray(feats, dtype=np.float32)[ok], lab[ok].astype(np.float32)


def train(feats, targs, steps: int = 3000, lr: float = 3e-3, seed: int = 0):
    w0 = init_weights(seed)
    w, loss, _ = S.snmf_mlp_train(feats, targs, w0, steps=steps, lr=lr)
    return w, loss


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--labels", choices=["greedy", "rollout"], default="rollout")
    ap.add_argument("--problems", type=int, default=400)
    ap.add_argument("--branches", type=int, default=2)
    ap.add_argument("--score", choices=["f", "pg"], default="f", help="rollout labels: objective or projected gradient")
    ap.add_argument("--margin", type=float, default=1e-12, help="rollout labels: relative margin over the plain step")
    ap.add_argument("--restarts", type=int, default=8)
    ap.add_argument("--per-traj", type=int, default=20)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    args = ap.parse_args(argv)
    t0 = time.time()
    if args.labels == "rollout":
        f, t = rollout_targets(*collect_rollout(args.problems, args.branches), score=args.score, margin=args.margin)
    else:
        f, t = collect(args.problems, args.restarts, args.per_traj)
    t1 = time.time()
    w, loss = train(f, t, args.steps, args.lr)
    t2 = time.time()
    hist = {str(v): int(np.sum(np.isclose(t, v))) for v in np.arange(-2.0, 2.01, 0.5)}
    base = float(np.mean((t - t.mean()) ** 2))
    rec = {"weights": [float(x) for x in w], "loss": loss, "target_variance": base, "samples": int(len(t)),
           "labels": args.labels if args.labels == "greedy" else f"rollout (score {args.score}, margin {args.margin:g})",
           "label_histogram": hist,
           "trajectories": args.problems * (args.branches if args.labels == "rollout" else args.restarts),
           "collect_seconds": t1 - t0, "train_seconds": t2 - t1, "steps": args.steps, "lr": args.lr,
           "distribution": "n~U{64..2048}, r~U{4..32}, 1% relative noise, FP32, penalty form, M=10",
           "problems": args.problems,
           "seed_base": TRAIN_SEED_BASE}
    json.dump(rec, open(args.out, "w"), indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "weights"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
