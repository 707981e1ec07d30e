"""Symmetric-half storage of a dense BF16 A (sym_half = 1; A symmetric, Sec. 1.2): only the
128 x 128 tiles on and above the diagonal are stored, and the tensor-core product reads a tile
below the diagonal as the transpose of its stored mirror.  Checked against the exact
emulation of the stored BF16 operands (the product), against the full-storage product on the
same handle options (the same BF16 values), and against the FP64 oracle's solve of the
headline workload (the solver end to end)."""
import json
import os

import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S

from gpu_helpers import rel
from test_gpu_bf16 import bf16_round

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _device_key():
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name}/{p.multi_processor_count}"


def _cache(path, key, **cfg):
    entry = dict(splits=0, stages=0, per_sm=0, bn=0, row_bm=0, ms=1.0)
    entry.update(cfg)
    json.dump({"format": "snmf-tune-1", "devices": {_device_key(): {key: entry}}}, open(path, "w"))
    return str(path)


def _apply(A, X, r, b, sym, cache):
    import torch
    dev = torch.device("cuda:0")
    o = S.snmf_default_options(precision=S.SNMF_BF16, batch=b, sym_half=sym, autotune=1 if cache else 0,
                               tune_cache=cache)
    h = S.snmf_create(S.dense_matrix(torch.tensor(A, device=dev)), r, o)
    try:
        Xt = torch.tensor(X, device=dev)
        Yt = torch.empty_like(Xt)
        xax = S.snmf_apply(h, Xt, Yt, X.shape[1])
    finally:
        S.snmf_destroy(h)
    return Yt.cpu().numpy().astype(np.float64), xax


@pytest.mark.parametrize("n,cols,cfg", [
    # 128-column tiles, 4 K slices, fused epilogue (r = 64): the headline's product shape
    (2048, 512, dict(splits=4, stages=2, per_sm=2, bn=128)),
    # a ragged n (last tile row and column partly beyond n), 3 slices whose last one ends past n
    (1000, 256, dict(splits=3, stages=2, per_sm=1, bn=256)),
    # r = 24 (no fused dots: the separate finish pass), 64-column tiles
    (1000, 192, dict(splits=2, stages=2, per_sm=2, bn=64)),
    # one slice over every K block of a row (rows of both kinds in one accumulation chain)
    (1024, 128, dict(splits=1, stages=4, per_sm=1, bn=128)),
    # 8 slices, K blocks of a slice crossing the diagonal
    (4096, 512, dict(splits=8, stages=3, per_sm=1, bn=128)),
])
def test_sym_half_product_matches_emulated_operands(tmp_path, n, cols, cfg):
    g = np.random.default_rng(7 * n + cols)
    B = g.random((n, n), dtype=np.float32)
    A = (B + B.T).astype(np.float32)
    X = g.random((n, cols), dtype=np.float32)
    At = bf16_round(A).astype(np.float64)
    Xh = bf16_round(X)
    Xl = bf16_round(X - Xh)
    ref = At @ (Xh.astype(np.float64) + Xl.astype(np.float64))
    r, b = cols // 8, 8
    Ys, xs = _apply(A, X, r, b, 1, _cache(tmp_path / "s.json", f"dense/bf16s/n{n}/r{r}/N{cols}", **cfg))
    Yf, xf = _apply(A, X, r, b, 0, _cache(tmp_path / "f.json", f"dense/bf16/n{n}/r{r}/N{cols}", **cfg))
    print(f"n {n} cols {cols} {cfg}: sym vs emulation {rel(Ys, ref):.2e}, full vs emulation {rel(Yf, ref):.2e}, "
          f"sym == full bitwise: {np.array_equal(Ys, Yf)}")
    assert rel(Ys, ref) <= 3e-5, rel(Ys, ref)
    assert np.max(np.abs(Ys - ref) / np.maximum(np.abs(ref), 1e-30)) <= 3e-5
    assert abs(xs - float(np.sum(X * ref))) <= 1e-5 * abs(xs)
    # the same BF16 values in the same K order: the two storages agree to FP32 rounding
    assert np.max(np.abs(Ys - Yf) / np.maximum(np.abs(Yf), 1e-30)) <= 1e-6


def test_sym_half_headline_solve_matches_oracle(tmp_path):
    """The headline workload at n = 2048 (BF16 A, r = 64, 8 restarts, lean learned step with the
    shipped weights, the bench's tile shapes) with A held as its upper tiles: every restart
    reaches relative projected gradient 1e-4 with its residual against the true A within 1e-3
    of the FP64 oracle's (tests/golden/oracle_dense2048_r64_b8.json), and the residual the
    solver reports (from ||A~||^2 of the stored tiles, off-diagonal tiles counted twice) agrees
    with the one computed here from the BF16-rounded A."""
    import torch
    from paper_2606_02887_gb300.train_controller import load_weights
    from workloads.configs import dense_planted_8192

    gold = json.load(open(os.path.join(GOLDEN, "oracle_dense2048_r64_b8.json")))
    n, r, b = gold["n"], gold["r"], gold["batch"]
    A, starts = dense_planted_8192(r, b, n=n)
    W0 = np.concatenate(starts, axis=1)
    dev = torch.device("cuda:0")
    cache = _cache(tmp_path / "tune.json", f"dense/bf16s/n{n}/r{r}/N{r * b}", splits=4, stages=2, per_sm=2,
                   bn=128, row_bm=64, row_tc=1)
    o = S.snmf_default_options(precision=S.SNMF_BF16, batch=b, max_iter=500, tol=1e-4, nonmonotone_M=10,
                               step_controller=3, autotune=1, tune_cache=cache, sym_half=1)
    h = S.snmf_create(S.dense_matrix(torch.tensor(A, dtype=torch.float32, device=dev)), r, o,
                      mlp_weights=load_weights())
    try:
        cfg = S.snmf_tuned_config(h)
        assert cfg["from_cache"] and (cfg["splits"], cfg["bn"]) == (4, 128)
        W = torch.tensor(W0, dtype=torch.float32, device=dev)
        H = W.clone()
        st, stats = S.snmf_solve(h, W, H)
        per = S.snmf_restart_stats(h, b)
    finally:
        S.snmf_destroy(h)
    assert st == S.SNMF_OK, stats
    Wn, Hn = W.cpu().numpy().astype(np.float64), H.cpu().numpy().astype(np.float64)
    nA = np.linalg.norm(A)
    Ab = bf16_round(A.astype(np.float32)).astype(np.float64)
    for j in range(b):
        sl = slice(j * r, (j + 1) * r)
        res = float(np.linalg.norm(A - Wn[:, sl] @ Hn[:, sl].T) / nA)
        ref = gold["restarts"][j]
        print("restart %d: residual %.6f (oracle %.6f), pg %.2e, iters %d (oracle %d)"
              % (j, res, ref["residual"], per["pg_rel"][j], per["iters"][j], ref["iters"]))
        assert ref["converged"]
        assert per["pg_rel"][j] <= 1e-4, (j, per["pg_rel"][j])
        assert abs(res - ref["residual"]) <= 1e-3, (j, res, ref["residual"])
    jb = stats["best_restart"]
    sl = slice(jb * r, (jb + 1) * r)
    res_b = float(np.linalg.norm(Ab - Wn[:, sl] @ Hn[:, sl].T) / np.linalg.norm(Ab))
    print(f"best restart {jb}: reported residual {stats['residual']:.8f}, from the BF16 A {res_b:.8f}")
    assert abs(stats["residual"] - res_b) <= 1e-3 * res_b
