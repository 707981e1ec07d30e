"""Training of the learned step controller on the GPU.

Data: record-mode solves (step_controller = 2) of seeded planted problems drawn like the
uneven-batch workload (n ~ U{64..2048}, r ~ U{4..32}, 1% relative noise), several random
restarts per problem in one batched solve.  At every inner step the solver follows the
plain BB trajectory and records the state's features and the best of 9 candidate
multipliers (the 1-step greedy label); about `per_traj` records per trajectory are kept.
Training: snmf_mlp_train (hand-written forward/backward and Adam kernels).

    python -m paper_2606_02887_gb300.train_controller --problems 1250 --restarts 8

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


def train(feats, targs, steps: int = 3000, lr: float = 3e-3, seed: int = 0):
    w0 = init_weights(seed)
    w, loss, _ = S.snmf_mlp_train(feats, targs, w0, steps=steps, lr=lr)
    return w, loss


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=1250)
    ap.add_argument("--restarts", type=int, default=8)
    ap.add_argument("--per-traj", type=int, default=20)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    args = ap.parse_args(argv)
    t0 = time.time()
    f, t = collect(args.problems, args.restarts, args.per_traj)
    t1 = time.time()
    w, loss = train(f, t, args.steps, args.lr)
    t2 = time.time()
    hist = {str(v): int(np.sum(np.isclose(t, v))) for v in np.arange(-2.0, 2.01, 0.5)}
    base = float(np.mean((t - t.mean()) ** 2))
    rec = {"weights": [float(x) for x in w], "loss": loss, "target_variance": base, "samples": int(len(t)),
           "trajectories": args.problems * args.restarts, "label_histogram": hist,
           "collect_seconds": t1 - t0, "train_seconds": t2 - t1, "steps": args.steps, "lr": args.lr,
           "distribution": "n~U{64..2048}, r~U{4..32}, 1% relative noise, FP32, penalty form, M=10",
           "seed_base": TRAIN_SEED_BASE}
    json.dump(rec, open(args.out, "w"), indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "weights"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
