"""Autotuner of the dense A*X product: the search picks a valid configuration, the JSON
cache keyed by device serves a second handle of the same shape, and tuned products agree
with the built-in configuration."""
import json
import math
import os

import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S
from workloads import planted_dense, uniform_init

from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def _apply(h, Xn):
    import torch
    X = torch.tensor(Xn, device="cuda:0")
    Y = torch.empty_like(X)
    S.snmf_apply(h, X, Y, Xn.shape[1])
    return Y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [S.SNMF_BF16, S.SNMF_F32])
def test_autotune_search_cache_and_agreement(tmp_path, prec):
    import torch
    n, r = 2048, 32
    A, _ = planted_dense(n, r, 0.05, seed=61 + prec)
    At = torch.tensor(A, dtype=torch.float32, device="cuda:0")
    cache = str(tmp_path / "tune.json")
    o = S.snmf_default_options(precision=prec, autotune=1, tune_cache=cache)
    h1 = S.snmf_create(S.dense_matrix(At), r, o)
    h0 = S.snmf_create(S.dense_matrix(At), r, S.snmf_default_options(precision=prec))
    try:
        c1 = S.snmf_tuned_config(h1)
        assert not c1["from_cache"] and c1["ms"] > 0 and c1["splits"] >= 1
        if prec == S.SNMF_BF16:
            assert c1["per_sm"] in (1, 2) and c1["stages"] >= 2
        data = json.load(open(cache))
        devs = data["devices"]
        assert len(devs) == 1
        key = f"dense/{'bf16' if prec == S.SNMF_BF16 else 'f32'}/n{n}/r{r}/N{r}"
        entry = next(iter(devs.values()))[key]
        assert entry["splits"] == c1["splits"]
        assert entry["row_bm"] in (0, 32, 64)
        assert (entry["bn"], entry["row_bm"]) == (c1["bn"], c1["row_bm"])
        h2 = S.snmf_create(S.dense_matrix(At), r, o)
        try:
            c2 = S.snmf_tuned_config(h2)
            assert c2["from_cache"] and {k: c2[k] for k in ("splits", "stages", "per_sm", "bn", "row_bm")} == \
                {k: c1[k] for k in ("splits", "stages", "per_sm", "bn", "row_bm")}
        finally:
            S.snmf_destroy(h2)
        Xn = np.random.default_rng(3).random((n, r)).astype(np.float32)
        # two correct accumulation orders of the same product (split counts chosen by timing).
        # FP32 CUDA cores: sums of n nonnegative terms in two orders differ by about sqrt(n) u
        # (u = 2^-24) relative; 8 sqrt(n) u = 2.2e-5 at n = 2048.  BF16 tensor cores: the FP32
        # accumulation drifts low in proportion to the K-chain length (a -5.7e-6 relative
        # rescaling over K = 8192, test_gpu_bf16.py), so different split counts differ by up
        # to that drift; the 3e-5 bar of the emulated-operand test holds for both.
        bar = 8.0 * math.sqrt(n) * 2.0 ** -24 if prec == S.SNMF_F32 else 3e-5
        assert rel(_apply(h1, Xn), _apply(h0, Xn)) <= bar
        with pytest.raises(S.SnmfError):
            S.snmf_tuned_config(h0)
    finally:
        S.snmf_destroy(h1)
        S.snmf_destroy(h0)
