"""Writes tests/golden/oracle_dense2048_r64_b8.json: the FP64 oracle's solve of each of the
8 restarts of the dense planted n = 2048, r = 64 workload (the n = 8192 recipe at n = 2048:
W0 ~ U[0,1], A = W0 W0^T + symmetric |N(0, 0.05^2)| noise, starts U[0, sqrt(mean(A)/r)]),
penalty form, nonmonotone memory 10, tolerance 1e-4, closed-form objective mode.  Per
restart: outer iterations, relative residual ||A - W Ht^T|| / ||A||, relative projected
gradient.  Calls only oracle/ and workloads/.  Restarts run in parallel processes.
Usage: python tests/golden/make_headline_oracle.py"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, R, B = 2048, 64, 8
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_dense{N}_r{R}_b{B}.json")


def solve(j):
    import oracle as O
    from workloads.configs import dense_planted_8192

    A, starts = dense_planted_8192(R, B, n=N)
    t = time.time()
    opts = O.Options(formulation="penalty", memory=10, max_iter=500, tol=1e-4, objective="closed")
    W, Ht, info = O.snmpbb_penalty(A, starts[j], starts[j], opts)
    return j, dict(iters=info["iters"], residual=info["residual"], pg_rel=info["pg"] / info["pg0"],
                   converged=bool(info["pg"] <= 1e-4 * info["pg0"]), f=info["f"], seconds=time.time() - t)


def main():
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(min(B, os.cpu_count() or 1)) as pool:
        res = dict(pool.map(solve, range(B)))
    data = {"n": N, "r": R, "batch": B,
            "options": "penalty, M=10, max_iter=500, tol=1e-4, lambda=0.01||A||_F, closed-form objective",
            "restarts": [res[j] for j in range(B)]}
    json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
    print(json.dumps(data, indent=1))


if __name__ == "__main__":
    main()
