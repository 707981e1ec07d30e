"""The dense planted workload at full size (n = 8192) over the rank sweep r in {16, 32, 64, 128,
256}, with A stored in BF16 and in FP32: each solve reaches relative projected gradient 1e-4 and
its residual against the true A is within 1e-3 of the FP64 oracle's solve from the same start
(tests/golden/oracle_iters_dense8192.json, written by make_oracle_iters.py from the oracle
alone).  The solver runs with its default tuning (the autotuner at create), as the bench does."""
import json
import os

import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_iters_dense8192.json")
RANKS = (16, 32, 64, 128, 256)


def _golden():
    return json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}


@pytest.mark.parametrize("precision", ["bf16", "f32"])
@pytest.mark.parametrize("r", RANKS)
def test_rank_sweep_full_size_matches_oracle(r, precision, tmp_path):
    import torch
    from workloads.configs import dense_planted_8192

    gold = _golden().get(str(r))
    if gold is None:
        pytest.skip(f"no oracle result for r = {r} in {os.path.basename(GOLDEN)}")
    assert gold["converged"]
    A, starts = dense_planted_8192(r)
    dev = torch.device("cuda:0")
    prec = S.SNMF_BF16 if precision == "bf16" else S.SNMF_F32
    o = S.snmf_default_options(precision=prec, batch=1, max_iter=500, tol=1e-4, nonmonotone_M=10, autotune=1,
                               tune_cache=str(tmp_path / "tune.json"))
    At = torch.tensor(A, dtype=torch.float32, device=dev)
    h = S.snmf_create(S.dense_matrix(At), r, o)
    try:
        W = torch.tensor(starts[0], dtype=torch.float32, device=dev)
        H = W.clone()
        st, stats = S.snmf_solve(h, W, H)
    finally:
        S.snmf_destroy(h)
    assert st == S.SNMF_OK, stats
    # residual against the true A, in FP64 on the device
    Ad = torch.tensor(A, dtype=torch.float64, device=dev)
    res = float(torch.linalg.norm(Ad - W.double() @ H.double().T) / torch.linalg.norm(Ad))
    print(f"r = {r} {precision}: residual {res:.6f} (oracle {gold['residual']:.6f}), pg {stats['pg_rel']:.2e}, "
          f"iterations {stats['iters']} (oracle {gold['iters']})")
    assert stats["pg_rel"] <= 1e-4
    assert abs(res - gold["residual"]) <= 1e-3, (res, gold["residual"])
