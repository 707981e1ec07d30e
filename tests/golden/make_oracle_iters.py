"""Writes tests/golden/oracle_iters_dense8192.json: the number of outer iterations the
FP64 oracle (penalty form, nonmonotone memory 10, closed-form objective mode) needs to
reach relative projected gradient 1e-4 on the n = 8192 planted workloads.  Calls only
oracle/ and workloads/.  Usage: python tests/golden/make_oracle_iters.py 64 [32 ...]"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from workloads.configs import dense_planted_8192  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iters_dense8192.json")


def main(rs):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for r in rs:
        A, starts = dense_planted_8192(r)
        t = time.time()
        opts = O.Options(formulation="penalty", memory=10, max_iter=500, tol=1e-4, objective="closed")
        W, Ht, info = O.snmpbb_penalty(A, starts[0], starts[0], opts)
        data[str(r)] = dict(iters=info["iters"], residual=info["residual"], pg_rel=info["pg"] / info["pg0"],
                            converged=bool(info["pg"] <= 1e-4 * info["pg0"]), seconds=time.time() - t,
                            options="penalty, M=10, max_iter=500, tol=1e-4, lambda=0.01||A||_F")
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
        print(r, data[str(r)], flush=True)


if __name__ == "__main__":
    main([int(x) for x in sys.argv[1:]] or [64])
